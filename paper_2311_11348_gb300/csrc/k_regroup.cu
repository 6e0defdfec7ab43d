// Grouping of the elements by polynomial order on the device (Sect. 3: the
// hierarchical basis makes an order change a change of which modes an
// element carries; the order-separated kernels want every order group
// contiguous).  Given the orders in the caller's element order, these
// kernels build everything that depends on them -- the internal permutation
// (a stable partition by order), the element and edge arrays in internal
// order, the correction edges grouped by the larger order of their two
// elements, and the offsets of the packed caller layout -- from the mesh
// arrays kept in the caller's order.  A context therefore changes orders
// (swe_set_orders, swe_adapt) without a host rebuild of its mesh.
//
// Stable partitions (elements by order, edges by correction group) are
// three passes over blocks of 256 units: per-block counts per category from
// warp ballots, one block scanning the counts, and a scatter that recomputes
// every unit's rank inside its block.  No atomics: the result is the same
// permutation a stable sort by category on the host gives.
#include "kernels.h"

namespace swedg {

namespace {

constexpr int RG_T = 256;  // units per block of the partition passes
constexpr int RG_W = RG_T / 32;
constexpr int RG_MAXC = 5;  // categories at most (orders 0..4)

// category of a unit: element u -> its order; edge i -> pmax - 2 for a
// correction edge (pmax = the larger order of its elements >= 2), else -1
struct ElemCat {
  const int8_t* p;
  __device__ int operator()(int64_t u) const { return p[u]; }
};
struct EdgeCat {
  const int8_t* p;  // orders, caller order
  const int32_t* eLu;
  const int32_t* eRu;
  __device__ int operator()(int64_t i) const {
    int pm = p[eLu[i]];
    const int r = eRu[i];
    if (r >= 0) pm = max(pm, (int)p[r]);
    return pm >= 2 ? pm - 2 : -1;
  }
};

// rank of this thread's unit among the units of its block with the same
// category (stable), and the block's counts per category in cnt_s
template <int NC>
__device__ __forceinline__ int block_rank(int cat, int (&cnt_s)[RG_W][RG_MAXC]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int rank = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const unsigned b = __ballot_sync(0xffffffffu, cat == c);
    if (cat == c) rank = __popc(b & lt);
    if (lane == 0) cnt_s[w][c] = __popc(b);
  }
  __syncthreads();
  if (cat >= 0)
    for (int v = 0; v < w; ++v) rank += cnt_s[v][cat];
  return rank;
}

template <int NC, typename Cat>
__global__ void __launch_bounds__(RG_T) k_part_counts(Cat cat, int64_t n, int32_t* cnt) {
  __shared__ int cnt_s[RG_W][RG_MAXC];
  const int64_t u = blockIdx.x * (int64_t)RG_T + threadIdx.x;
  const int c = u < n ? cat(u) : -1;
  block_rank<NC>(c, cnt_s);
  if (threadIdx.x < NC) {
    int s = 0;
    for (int v = 0; v < RG_W; ++v) s += cnt_s[v][threadIdx.x];
    cnt[(int64_t)blockIdx.x * NC + threadIdx.x] = s;
  }
}

// one block: off[b][c] = start[c] + sum_{b' < b} cnt[b'][c], start[c] = sum
// of the totals of the categories before c (start[NC] = their sum)
template <int NC>
__global__ void __launch_bounds__(1024) k_part_scan(const int32_t* cnt, int64_t nblk, int64_t* off, int64_t* start) {
  __shared__ int64_t part[1024][RG_MAXC];
  __shared__ int64_t base[RG_MAXC + 1];
  const int t = threadIdx.x;
  const int64_t per = (nblk + 1023) / 1024, b0 = t * per, b1 = min(nblk, b0 + per);
  int64_t s[RG_MAXC] = {0, 0, 0, 0, 0};
  for (int64_t b = b0; b < b1; ++b)
    for (int c = 0; c < NC; ++c) s[c] += cnt[b * NC + c];
  for (int c = 0; c < NC; ++c) part[t][c] = s[c];
  __syncthreads();
  if (t < NC) {  // exclusive scan over the threads' segments, per category
    int64_t acc = 0;
    for (int v = 0; v < 1024; ++v) {
      const int64_t x = part[v][t];
      part[v][t] = acc;
      acc += x;
    }
    base[t] = acc;  // the category's total, for now
  }
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int c = 0; c < NC; ++c) {
      const int64_t x = base[c];
      base[c] = acc;
      start[c] = acc;
      acc += x;
    }
    start[NC] = acc;
  }
  __syncthreads();
  int64_t run[RG_MAXC];
  for (int c = 0; c < NC; ++c) run[c] = base[c] + part[t][c];
  for (int64_t b = b0; b < b1; ++b)
    for (int c = 0; c < NC; ++c) {
      off[b * NC + c] = run[c];
      run[c] += cnt[b * NC + c];
    }
}

// elements: perm[e] = u, inv[u] = e, p_int[e] = p_u for the new internal index e
__global__ void __launch_bounds__(RG_T) k_elem_scatter(const int8_t* p_user, int64_t ne, const int64_t* off,
                                                      int32_t* perm, int32_t* inv, int8_t* p_int) {
  __shared__ int cnt_s[RG_W][RG_MAXC];
  const int64_t u = blockIdx.x * (int64_t)RG_T + threadIdx.x;
  const int c = u < ne ? p_user[u] : -1;
  const int r = block_rank<5>(c, cnt_s);
  if (u < ne) {
    const int64_t e = off[(int64_t)blockIdx.x * 5 + c] + r;
    perm[e] = (int32_t)u;
    inv[u] = (int32_t)e;
    p_int[e] = (int8_t)c;
  }
}

// edges: slot[i] = (pmax << 28) | position in its correction group, or -1;
// lists[(pmax - 2) * nedge + position] = i.  off includes the group starts
// (start3), which the positions are taken relative to.
__global__ void __launch_bounds__(RG_T) k_edge_scatter(EdgeCat cat, int64_t nedge, const int64_t* off,
                                                      const int64_t* start3, int32_t* slot, int32_t* lists) {
  __shared__ int cnt_s[RG_W][RG_MAXC];
  const int64_t i = blockIdx.x * (int64_t)RG_T + threadIdx.x;
  const int c = i < nedge ? cat(i) : -1;
  const int r = block_rank<3>(c, cnt_s);
  if (i < nedge) {
    if (c < 0) {
      slot[i] = -1;
    } else {
      const int64_t pos = off[(int64_t)blockIdx.x * 3 + c] + r - start3[c];
      slot[i] = ((c + 2) << 28) | (int32_t)pos;
      lists[(int64_t)c * nedge + pos] = (int32_t)i;
    }
  }
}

// element and edge arrays in the new internal order
__global__ void k_gather_elems(MeshStatic S, const int32_t* __restrict__ perm, DevMeshOut D) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ne = S.ne;
  if (e >= ne) return;
  const int64_t u = perm[e];
#pragma unroll 4
  for (int r = 0; r < NGEO; ++r) {
    const double v = S.geo_u[r * ne + u];
    D.geo[r * ne + e] = v;
    D.geo32[r * ne + e] = (float)v;
  }
  const double2* src = reinterpret_cast<const double2*>(S.etb_u + 12 * u);
  double2* dst = reinterpret_cast<double2*>(D.etb + 12 * e);
#pragma unroll
  for (int k = 0; k < 6; ++k) dst[k] = src[k];
  D.mem[e] = S.mem_u[u];
#pragma unroll
  for (int k = 0; k < 3; ++k) D.eedge[k * ne + e] = S.eedge_u[k * ne + u];
}

__global__ void k_gather_edges(MeshStatic S, const int32_t* __restrict__ inv, DevMeshOut D) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= S.nedge) return;
  D.eL[i] = inv[S.eLu[i]];
  const int32_t r = S.eRu[i];
  D.eR[i] = r >= 0 ? inv[r] : -1;
}

// packed caller layout: off[u] = sum_{u' < u} 3 K(p_u'), total in *total
__global__ void __launch_bounds__(RG_T) k_packed_counts(const int8_t* p_user, int64_t ne, int64_t* bsum) {
  __shared__ int64_t s[RG_T];
  const int64_t u = blockIdx.x * (int64_t)RG_T + threadIdx.x;
  s[threadIdx.x] = u < ne ? 3 * Kof(p_user[u]) : 0;
  __syncthreads();
  for (int w = RG_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(RG_T) k_packed_offsets(const int8_t* p_user, int64_t ne, const int64_t* boff,
                                                        int64_t* off) {
  __shared__ int64_t s[RG_T];
  const int64_t u = blockIdx.x * (int64_t)RG_T + threadIdx.x;
  const int64_t v = u < ne ? 3 * Kof(p_user[u]) : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = 1; w < RG_T; w <<= 1) {  // inclusive Hillis-Steele scan
    const int64_t x = threadIdx.x >= w ? s[threadIdx.x - w] : 0;
    __syncthreads();
    s[threadIdx.x] += x;
    __syncthreads();
  }
  if (u < ne) off[u] = boff[blockIdx.x] + s[threadIdx.x] - v;
}

// one block: exclusive scan of the block sums; total in out[nblk]
__global__ void __launch_bounds__(1024) k_scan_blocks(const int64_t* bsum, int64_t nblk, int64_t* out) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nblk + 1023) / 1024, b0 = t * per, b1 = min(nblk, b0 + per);
  int64_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += bsum[b];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t acc = 0;
    for (int v = 0; v < 1024; ++v) {
      const int64_t x = part[v];
      part[v] = acc;
      acc += x;
    }
    out[nblk] = acc;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t b = b0; b < b1; ++b) {
    out[b] = run;
    run += bsum[b];
  }
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int64_t regroup_blocks(int64_t n) { return nb(n, RG_T); }

int launch_regroup(cudaStream_t s, const MeshStatic& S, const int8_t* p_user, DevMeshOut D, RegroupScratch W) {
  const int64_t ne = S.ne, nE = S.nedge;
  const int64_t be = nb(ne, RG_T), bg = nb(nE, RG_T);
  // W.info: [0..5] order group starts, [6..9] correction edge group starts, [10] packed size
  k_part_counts<5><<<(unsigned)be, RG_T, 0, s>>>(ElemCat{p_user}, ne, W.ecnt);
  k_part_scan<5><<<1, 1024, 0, s>>>(W.ecnt, be, W.eoff, W.info);
  k_elem_scatter<<<(unsigned)be, RG_T, 0, s>>>(p_user, ne, W.eoff, D.perm, D.inv, D.p);
  count_launch(3);
  if (nE > 0) {
    const EdgeCat ec{p_user, S.eLu, S.eRu};
    k_part_counts<3><<<(unsigned)bg, RG_T, 0, s>>>(ec, nE, W.gcnt);
    k_part_scan<3><<<1, 1024, 0, s>>>(W.gcnt, bg, W.goff, W.info + 6);
    k_edge_scatter<<<(unsigned)bg, RG_T, 0, s>>>(ec, nE, W.goff, W.info + 6, D.slot, D.lists);
    k_gather_edges<<<nb(nE, 256), 256, 0, s>>>(S, D.inv, D);
    count_launch(4);
  }
  k_gather_elems<<<nb(ne, 256), 256, 0, s>>>(S, D.perm, D);
  k_packed_counts<<<(unsigned)be, RG_T, 0, s>>>(p_user, ne, W.psum);
  k_scan_blocks<<<1, 1024, 0, s>>>(W.psum, be, W.poff);
  k_packed_offsets<<<(unsigned)be, RG_T, 0, s>>>(p_user, ne, W.poff, D.off);
  count_launch(4);
  SWE_CUDA_OK(cudaGetLastError());
  // the packed total (poff[be]) next to the group starts
  SWE_CUDA_OK(cudaMemcpyAsync(W.info + 10, W.poff + be, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  return 0;
}

}  // namespace swedg
