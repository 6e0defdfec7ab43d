// Base part of the order-separated scheme (Sect. 3): every term whose test
// index and coefficient indices are modes of degree <= 1, on every element,
// in FP64.  Plus the layout conversions, the CFL reduction, the time update
// and the diagnostics.
//
// Kernels (one thread per element or per edge, FP64-pipe bound on GB300):
//   k_usolve_base  auxiliary system uH = q (Sect. 3) for p <= 1 elements
//                  (and, in the first stage of a step, the CFL bounds of its
//                  elements: min over elements, exact, order independent)
//   k_edge_base    Lax-Friedrichs flux (Sect. 2) of the P1 traces at the two
//                  Gauss points of every edge, lambda of Eq. (10) from means
//   k_elem_base    volume + source terms (Eq. 13 with the degree-1 tensors in
//                  closed form), edge projections, correction merge and the
//                  SSP-RK stage combination of the base modes
#include <cfloat>

#include "kernels.h"
#include "tables.h"


namespace swedg {

__constant__ double cTs[6];  // T[1][1][1], T[2][1][1], T[1][1][2], T[2][1][2], T[1][2][2], T[2][2][2] over phihat_1

void upload_base_tables() {
  const RefTables& R = tables();
  const double Ts[6] = {R.T[1][1][1] / R.phi0, R.T[2][1][1] / R.phi0, R.T[1][1][2] / R.phi0,
                        R.T[2][1][2] / R.phi0, R.T[1][2][2] / R.phi0, R.T[2][2][2] / R.phi0};
  cudaMemcpyToSymbol(cTs, Ts, sizeof Ts);
}

static inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Grid of the FP64-pipe-bound base kernels: `per_sm` resident blocks per SM,
// grid-stride loops over the work.  A few warps per SM already keep the FP64
// pipe busy; the rest of the SM stays free for the concurrent FP32 correction.
static int g_sm_count = 152;
void set_sm_count(int n) { g_sm_count = n > 0 ? n : 152; }
static inline int capped_blocks(int64_t n, int t, int per_sm) {
  const int64_t b = (n + t - 1) / t, cap = (int64_t)g_sm_count * per_sm;
  return (int)(per_sm <= 0 || b < cap ? b : cap);
}

template <typename T>
__device__ __forceinline__ T* chp(void* p) { return reinterpret_cast<T*>(p); }

// Work distribution of the persistent base kernels over n units (edges or
// elements).  chunk == 0 or work == nullptr: equal grid-stride shares.
// Otherwise every block takes tiles of chunk * blockDim.x consecutive units
// from an atomic ticket counter (work[0]) until none are left -- the next
// ticket is fetched while the current tile runs -- so a block on an SM that
// the concurrent correction kernels keep busy simply takes fewer tiles; the
// last block to finish (counted in work[1]) resets both counters for the next
// launch on the stream.  Every unit is computed by one thread with the same
// arithmetic whatever the schedule, so results do not depend on it.
template <typename F>
__device__ __forceinline__ void for_units(int64_t n, int chunk, unsigned* work, F&& f) {
  const bool dyn = chunk > 0 && work != nullptr;
  __shared__ unsigned s_ticket;
  const int64_t tile = dyn ? (int64_t)chunk * blockDim.x : (int64_t)gridDim.x * blockDim.x;
  const int64_t ntiles = (n + tile - 1) / tile;
  // static: tile t is the t-th grid-wide stride, every block takes each t
  // with its own offset blockIdx.x * blockDim.x; dynamic: tile t is chunk *
  // blockDim.x consecutive units, taken from the ticket counter
  int64_t t = 0;
  if (dyn) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(work, 1u);
    __syncthreads();
    t = s_ticket;
  }
  const int64_t off = dyn ? threadIdx.x : blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per = dyn ? chunk : 1;
#pragma unroll 1
  while (t < ntiles) {
    if (dyn) {
      __syncthreads();  // every thread has read the ticket
      if (threadIdx.x == 0) s_ticket = atomicAdd(work, 1u);
    }
    const int64_t base = t * tile + off;
#pragma unroll 1
    for (int k = 0; k < per; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x;
      if (i < n) f(i);
    }
    if (dyn) {
      __syncthreads();  // the next ticket has arrived
      t = s_ticket;
    } else {
      ++t;
    }
  }
  if (dyn && threadIdx.x == 0) {
    // this block takes no more tickets; the last one out resets the counters
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
      work[0] = 0u;
      work[1] = 0u;
      __threadfence();
    }
  }
}

// ---------------------------------------------------------------------------
// layout conversion: caller layout <-> internal state.  Caller layouts: the
// full c[3][15][ne_user] (off == nullptr), or packed element by element,
// element u's 3 K(p_u) values (field-major) from off[u] (modes < K(p_u) only).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t user_at(const int64_t* off, int64_t ne, int64_t u, int K, int f, int i) {
  return off ? off[u] + f * K + i : (f * KMAX + i) * ne + u;
}

template <typename TC>
__global__ void k_from_user(DevMesh m, Groups G, const int32_t* perm, const int64_t* off,
                            const double* __restrict__ cu, StateDev st) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int64_t ne = m.ne, u = perm[e];
  const int p = m.p[e], K = Kof(p);
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < 3; ++i) {
      const double v = i < K ? cu[user_at(off, ne, u, K, f, i)] : 0.0;
      st.cb[(f * 3 + i) * ne + e] = v;
      if (st.cb32) st.cb32[(f * 3 + i) * ne + e] = (float)v;
    }
  if (p >= 2) {
    const int64_t n = G.start[p + 1] - G.start[p], l = e - G.start[p];
    TC* h = chp<TC>(st.ch[p]);
    for (int f = 0; f < 3; ++f)
      for (int i = 3; i < K; ++i) h[(f * (K - 3) + (i - 3)) * n + l] = (TC)cu[user_at(off, ne, u, K, f, i)];
  }
}

template <typename TC>
__global__ void k_to_user(DevMesh m, Groups G, const int32_t* perm, const int64_t* off, StateDev st,
                          double* __restrict__ cu) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int64_t ne = m.ne, u = perm[e];
  const int p = m.p[e], K = Kof(p);
  const int KO = off ? K : KMAX;  // the packed layout holds the modes < K only
  for (int f = 0; f < 3; ++f) {
    for (int i = 0; i < 3 && i < KO; ++i) cu[user_at(off, ne, u, K, f, i)] = i < K ? st.cb[(f * 3 + i) * ne + e] : 0.0;
    for (int i = 3; i < KO; ++i) {
      double v = 0.0;
      if (i < K) {
        const int64_t n = G.start[p + 1] - G.start[p], l = e - G.start[p];
        v = (double)chp<TC>(st.ch[p])[(f * (K - 3) + (i - 3)) * n + l];
      }
      cu[user_at(off, ne, u, K, f, i)] = v;
    }
  }
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                      int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

int launch_sub(cudaStream_t s, const double* a, const double* b, double* out, int64_t n) {
  if (n == 0) return 0;
  k_sub<<<nblocks(n, 256), 256, 0, s>>>(a, b, out, n);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_from_user(cudaStream_t s, const DevMesh& m, const Groups& G, const int32_t* perm, const int64_t* off,
                     int corr_fp32, const double* cu, StateDev st) {
  if (m.ne == 0) return 0;
  if (corr_fp32) k_from_user<float><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, perm, off, cu, st);
  else k_from_user<double><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, perm, off, cu, st);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_to_user(cudaStream_t s, const DevMesh& m, const Groups& G, const int32_t* perm, const int64_t* off,
                   int corr_fp32, StateDev st, double* cu) {
  if (m.ne == 0) return 0;
  if (corr_fp32)
    k_to_user<float><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, perm, off, st, cu);
  else
    k_to_user<double><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, perm, off, st, cu);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------------------
// auxiliary system for p <= 1 (Sect. 3):  M_H u = U, M_H v = V with
//   M_H[i][j] = (1/s) sum_{n < K(i,j)} H_n T[n][i][j],  K(1,1) = 1, else 3.
// The 3 x 3 symmetric system is solved with its adjugate (one division).
// The basis is orthonormal with the constant phihat_1, so T[0][i][j] =
// T[i][0][j] = phihat_1 delta_ij: over phihat_1 the first row and column are
// H_0, H_1, H_2 and the other entries need the six T[n][i][j] with n, i, j
// >= 1 only (the factor comes back in the final scale).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_usolve_base(DevMesh m, int64_t n_end, Phys ph, const double* __restrict__ cb,
                                                     double* __restrict__ ub, float* __restrict__ ub32,
                                                     unsigned* status, unsigned long long* dmin) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dcfl = DBL_MAX;
  int mem = 0;
  if (e < n_end) {
    const int64_t ne = m.ne;
    const double rs = m.geo[G_RS * ne + e];
    const double H0 = cb[0 * ne + e] + m.geo[G_HB0 * ne + e];
    const double U0 = cb[3 * ne + e], V0 = cb[6 * ne + e];
    if (!(H0 * m.geo[G_M0 * ne + e] > ph.h_min)) {  // mean depth: mode 0 times phi_{e,1} = phihat_1 / s_e
      atomicOr(status, (unsigned)ST_DEPTH);
      atomicOr(m.mstatus + m.mem[e], (unsigned)ST_DEPTH);
    }
    double v[6];
    if (m.p[e] == 0) {
      const double r = 1.0 / (H0 * m.geo[G_M0 * ne + e]);
      v[0] = U0 * r; v[1] = 0.0; v[2] = 0.0;
      v[3] = V0 * r; v[4] = 0.0; v[5] = 0.0;
    } else {
      const double H1 = cb[1 * ne + e] + m.geo[G_HB1 * ne + e];
      const double H2 = cb[2 * ne + e] + m.geo[G_HB2 * ne + e];
      const double U1 = cb[4 * ne + e], U2 = cb[5 * ne + e];
      const double V1 = cb[7 * ne + e], V2 = cb[8 * ne + e];
      // entries of S / phihat_1 with S = s M (the 1/s factor cancels in the
      // adjugate solve up to a final scale)
      const double a = H0, b = H1, c = H2;
      const double d = H0 + H1 * cTs[0] + H2 * cTs[1];
      const double f = H1 * cTs[2] + H2 * cTs[3];
      const double h = H0 + H1 * cTs[4] + H2 * cTs[5];
      // M = (phihat_1 / s) [[a b c][b d f][c f h]];  u = s adj(S') U / (phihat_1 det(S'))
      const double C00 = d * h - f * f, C01 = c * f - b * h, C02 = b * f - c * d;
      const double C11 = a * h - c * c, C12 = b * c - a * f, C22 = a * d - b * b;
      const double det = a * C00 + b * C01 + c * C02;
      const double r = 1.0 / (det * m.geo[G_M0 * ne + e]);
      v[0] = (C00 * U0 + C01 * U1 + C02 * U2) * r; v[1] = (C01 * U0 + C11 * U1 + C12 * U2) * r;
      v[2] = (C02 * U0 + C12 * U1 + C22 * U2) * r; v[3] = (C00 * V0 + C01 * V1 + C02 * V2) * r;
      v[4] = (C01 * V0 + C11 * V1 + C12 * V2) * r; v[5] = (C02 * V0 + C12 * V1 + C22 * V2) * r;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      ub[i * ne + e] = v[i];
      if (ub32) ub32[i * ne + e] = (float)v[i];
    }
    if (dmin) {
      mem = m.mem[e];
      dcfl = cfl_bound(v[0], v[3], H0, rs, ph.g, m.geo[G_DIAM * ne + e], m.p[e]);
    }
  }
  if (dmin) cfl_min_store(dmin, mem, dcfl);  // uniform over the grid: every lane of the warp is here
}

int launch_usolve_base(cudaStream_t s, const DevMesh& m, const Groups& G, const Phys& ph, const double* cb,
                       double* ub, float* ub32, unsigned* status, unsigned long long* dmin) {
  const int64_t n = G.start[2];
  if (n == 0) return 0;
  const int ut = launch_shape().usolve_threads;
  k_usolve_base<<<nblocks(n, ut), ut, 0, s>>>(m, n, ph, cb, ub, ub32, status, dmin);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

__global__ void k_reset_min(unsigned long long* dmin, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dmin[i] = (unsigned long long)__double_as_longlong(DBL_MAX);
}

int launch_reset_min(cudaStream_t s, unsigned long long* dmin, int nmem) {
  k_reset_min<<<nblocks(nmem, 128), 128, 0, s>>>(dmin, nmem);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// per member: dt = dt_fixed > 0 ? dt_fixed : cfl * min (before the step), and
// the minimum back to DBL_MAX for the next step's reduction (the velocity
// solves of the first stage fold their elements' CFL bounds into it);
// t += dt (after the step)
__global__ void k_set_dt(double* dt_dev, unsigned long long* dmin, double cfl, double dt_fixed, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    dt_dev[i] = dt_fixed > 0.0 ? dt_fixed : cfl * __longlong_as_double((long long)dmin[i]);
    dmin[i] = (unsigned long long)__double_as_longlong(DBL_MAX);
  }
}
__global__ void k_fill(double* p, double v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

int launch_fill(cudaStream_t s, double* p, double v, int n) {
  if (n <= 0) return 0;
  k_fill<<<nblocks(n, 128), 128, 0, s>>>(p, v, n);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

__global__ void k_advance_time(double* t_dev, const double* dt_dev, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t_dev[i] += dt_dev[i];
}

int launch_advance_time(cudaStream_t s, double* t_dev, unsigned long long* dmin, double cfl, double dt_fixed,
                        double* dt_dev, int nmem) {
  if (t_dev == nullptr) k_set_dt<<<nblocks(nmem, 128), 128, 0, s>>>(dt_dev, dmin, cfl, dt_fixed, nmem);
  else k_advance_time<<<nblocks(nmem, 128), 128, 0, s>>>(t_dev, dt_dev, nmem);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

__device__ __forceinline__ double tide_value(const Phys& ph, double t) {
  if (ph.tide_period <= 0.0) return ph.tide_amp;
  return ph.tide_amp * sin(2.0 * 3.14159265358979323846 * t / ph.tide_period + ph.tide_phase);
}

// ---------------------------------------------------------------------------
// Base edge flux.  For the P1 parts of both sides: traces at the two Gauss
// points, the LF flux (Sect. 2)
//   A_hat = 1/2 ((A(c) + A(c+)).n + lambda (c - c+)),
//   A.n = (q.n,  U (u.n) + g nx (xi^2/2 + xi h_b),  V (u.n) + g ny (...)),
// with lambda from the element means (Eq. 10, Sect. 3), stored pre-weighted
// by |E| w_g at the points in the left element's direction.
// ---------------------------------------------------------------------------
// Traces of xi, U, V and w = u.n (P1 parts) of one side at the two Gauss
// points.  Mode 1 is the constant sqrt 2 on every edge, so its trace is shared.
struct Tr2 { double xi[2], U[2], V[2], w[2]; double xi0, w0; };

// P1 traces of one side at the two points of the base rule (edge direction of
// the left element), from the scaled basis table: no FP64 multiply for the
// basis values.  w is u . (|E| w_g / 2) n, the weighted normal velocity.
__device__ __forceinline__ void p1_traces(const DevMesh& m, const double* __restrict__ cb,
                                          const double* __restrict__ ub, int64_t ne, int64_t e, int k, bool reverse,
                                          double nxw, double nyw, Tr2& t) {
  const double m0 = m.geo[G_M0 * ne + e];
  const double2 p0 = *reinterpret_cast<const double2*>(m.etb + (3 * e + k) * 4);
  const double2 p1 = *reinterpret_cast<const double2*>(m.etb + (3 * e + k) * 4 + 2);
  const double b10 = reverse ? p1.x : p0.x, b20 = reverse ? p1.y : p0.y;
  const double b11 = reverse ? p0.x : p1.x, b21 = reverse ? p0.y : p1.y;
  double c[3][3], w[3];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int i = 0; i < 3; ++i) c[f][i] = cb[(f * 3 + i) * ne + e];
#pragma unroll
  for (int i = 0; i < 3; ++i) w[i] = ub[i * ne + e] * nxw + ub[(3 + i) * ne + e] * nyw;
  double* out[3] = {t.xi, t.U, t.V};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const double a0 = c[f][0] * m0;
    out[f][0] = a0 + c[f][1] * b10 + c[f][2] * b20;
    out[f][1] = a0 + c[f][1] * b11 + c[f][2] * b21;
    if (f == 0) t.xi0 = a0;
  }
  t.w0 = w[0] * m0;
  t.w[0] = t.w0 + w[1] * b10 + w[2] * b20;
  t.w[1] = t.w0 + w[1] * b11 + w[2] * b21;
}

__global__ void __launch_bounds__(128) k_edge_base(DevMesh m, Phys ph, Stage stg, const double* __restrict__ cb,
                                                   const double* __restrict__ ub, double* __restrict__ Fb, int chunk,
                                                   unsigned* work) {
  for_units(m.nedge, chunk, work, [&](int64_t ed) {
  const int64_t ne = m.ne, nE = m.nedge;
  const int L = m.eL[ed], R = m.eR[ed], info = m.einfo[ed];
  const int kL = info & 3, kR = (info >> 2) & 3, bc = info >> 4;
  // the flux comes out weighted by wl = |E| w_g / 2 through the weighted
  // normal (nxw, nyw) = wl n, which also weights w = u.n and so lambda
  const double nxw = m.egeo[E_NXW * nE + ed], nyw = m.egeo[E_NYW * nE + ed];
  const double hmid = m.egeo[E_HMID * nE + ed];
  Tr2 a, b;
  p1_traces(m, cb, ub, ne, L, kL, false, nxw, nyw, a);
  const double unL = a.w0, HL = a.xi0 + hmid;
  double unR, HR;
  if (R >= 0) {
    p1_traces(m, cb, ub, ne, R, kR, true, nxw, nyw, b);
    unR = b.w0;
    HR = b.xi0 + hmid;
  } else if (bc == 2) {
    const double xh = tide_value(ph, stage_time(stg, m.emem[ed]));
    b = a;
    b.xi[0] = xh; b.xi[1] = xh;
    unR = unL;
    HR = xh + hmid;
  } else {
    // mirror state: q+ = q - 2 (q.n) n, (u.n)+ = -(u.n), xi+ = xi
    const double nx = m.egeo[E_NX * nE + ed], ny = m.egeo[E_NY * nE + ed];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const double qn2 = -2.0 * (a.U[g] * nx + a.V[g] * ny);
      b.xi[g] = a.xi[g];
      b.U[g] = a.U[g] + qn2 * nx;
      b.V[g] = a.V[g] + qn2 * ny;
      b.w[g] = -a.w[g];
    }
    unR = -unL;
    HR = HL;
  }
  // lambda of Eq. (10) from the means (Sect. 3); max sqrt = sqrt max; times wl
  const double wl = m.egeo[E_WLEN * nE + ed];
  const double lam = fmax(fabs(unL), fabs(unR)) + wl * sqrt(ph.g * fmax(HL, HR));
  // momentum rows as U (w + lambda) + U+ (w+ - lambda) + P n: the two
  // factors are shared by both rows
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const double hb = m.egeo[(E_HG0 + g) * nE + ed];
    const double P = ph.g * (a.xi[g] * (0.5 * a.xi[g] + hb) + b.xi[g] * (0.5 * b.xi[g] + hb));
    const double wa = a.w[g] + lam, wb = b.w[g] - lam;
    Fb[(0 * 2 + g) * nE + ed] = (a.U[g] + b.U[g]) * nxw + (a.V[g] + b.V[g]) * nyw + lam * (a.xi[g] - b.xi[g]);
    Fb[(1 * 2 + g) * nE + ed] = a.U[g] * wa + b.U[g] * wb + P * nxw;
    Fb[(2 * 2 + g) * nE + ed] = a.V[g] * wa + b.V[g] * wb + P * nyw;
  }
  });
}

// the tile size of the dynamic schedule, 0 for the static one (an uncapped
// grid of one block per base_threads units needs no schedule)
static inline int base_chunk(const LaunchShape& L) { return L.base_bpsm > 0 ? L.base_chunk : 0; }

int launch_edge_base(cudaStream_t s, const DevMesh& m, const Phys& ph, const Stage& stg, const double* cb,
                     const double* ub, EdgeFlux fx, unsigned* work) {
  if (m.nedge == 0) return 0;
  const LaunchShape& L = launch_shape();
  k_edge_base<<<capped_blocks(m.nedge, L.base_threads, L.base_bpsm), L.base_threads, 0, s>>>(m, ph, stg, cb, ub, fx.Fb,
                                                                                             base_chunk(L), work);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------------------
// Base element update.  For test modes q of degree 1, grad phi_q is constant,
// so by orthonormality (Eq. 13 restricted to indices <= 3)
//   (A_xi, grad phi_q) = grad phi_q . (U_1, V_1) sqrt|Omega|
//   (A_U , grad phi_q) = d_x phi_q sum_i (U_i u_i + g(xi_i^2/2 + xi_i hb_i))
//                      + d_y phi_q sum_i U_i v_i          (and alike for V),
// the source (r, phi_q) = g grad h_b xi_q (- tau u_q + f_c V_q, - tau v_q -
// f_c U_q with bottom friction and Coriolis), and the edge terms are
// -sum_g F_g phi_q(x_g) over the three edges (sign flipped for the right side).
// ---------------------------------------------------------------------------
// MINB: blocks per SM the register allocation must allow -- 4 (128 registers)
// for uncapped grids, where the kernel's own occupancy is what counts; 3 for
// grids capped at a few blocks per SM beside the correction kernels, where
// the measured step is faster with the unrestricted allocation
template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_elem_base(DevMesh m, Phys ph, Stage stg, const double* __restrict__ cbS,
                                                   const double* __restrict__ cbN, double* __restrict__ cbO,
                                                   float* __restrict__ cbO32, const double* __restrict__ ub,
                                                   const double* __restrict__ Fb, const double* __restrict__ Fbc,
                                                   const double* __restrict__ rc, int64_t rc_start, int chunk,
                                                   unsigned* work) {
  const int64_t ne = m.ne, nE = m.nedge;
  const double* geo = m.geo;
  for_units(ne, chunk, work, [&](int64_t e) {
  double c[3][3], u[2][3];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int i = 0; i < 3; ++i) c[f][i] = cbS[(f * 3 + i) * ne + e];
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int i = 0; i < 3; ++i) u[f][i] = ub[(f * 3 + i) * ne + e];
  const double rs = geo[G_RS * ne + e], sqa = geo[G_SQA * ne + e], m0 = geo[G_M0 * ne + e];
  const double hb[3] = {geo[G_HB0 * ne + e], geo[G_HB1 * ne + e], geo[G_HB2 * ne + e]};
  double r[3][3];
  // volume terms
  double Axx = 0.0, Axy = 0.0, Ayx = 0.0, Ayy = 0.0, P = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Axx += c[1][i] * u[0][i]; Axy += c[1][i] * u[1][i];
    Ayx += c[2][i] * u[0][i]; Ayy += c[2][i] * u[1][i];
    P += c[0][i] * (0.5 * c[0][i] + hb[i]);
  }
  P *= ph.g;
  Axx += P;
  Ayy += P;
  const double gdx = geo[G_GDHX * ne + e], gdy = geo[G_GDHY * ne + e];
  const double U0s = c[1][0] * sqa, V0s = c[2][0] * sqa;
  r[0][0] = 0.0;
  r[1][0] = gdx * c[0][0];
  r[2][0] = gdy * c[0][0];
#pragma unroll
  for (int q = 1; q < 3; ++q) {
    const double gx = geo[(q == 1 ? G_GQ1X : G_GQ2X) * ne + e], gy = geo[(q == 1 ? G_GQ1Y : G_GQ2Y) * ne + e];
    r[0][q] = gx * U0s + gy * V0s;
    r[1][q] = gx * Axx + gy * Axy + gdx * c[0][q];
    r[2][q] = gx * Ayx + gy * Ayy + gdy * c[0][q];
  }
  if (ph.src) {
    // bottom friction and Coriolis of Eq. (5); tau from the element means of H
    // and u (Sect. 3), mean = mode 0 / sqrt|Omega| = mode 0 * sqrt 2 / s_e
    const double ra = 1.4142135623730951 * rs;
    const double Hm = (c[0][0] + hb[0]) * ra, um = u[0][0] * ra, vm = u[1][0] * ra;
    const double tau = ph.fric_lin * Hm + ph.fric_quad * sqrt(um * um + vm * vm);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      r[1][q] += ph.f_c * c[2][q] - tau * u[0][q];
      r[2][q] -= ph.f_c * c[1][q] + tau * u[1][q];
    }
  }
  // edge terms
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int ee = m.eedge[k * ne + e];
    const int64_t ed = ee >> 1;
    const bool right = ee & 1;
    double F[3][2];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      F[f][0] = Fb[(f * 2 + 0) * nE + ed];
      F[f][1] = Fb[(f * 2 + 1) * nE + ed];
      if (!stg.base_only) {
        F[f][0] += Fbc[(f * 2 + 0) * nE + ed];
        F[f][1] += Fbc[(f * 2 + 1) * nE + ed];
      }
    }
    // the basis at the edge's two points, times -1/s_e (left side) or +1/s_e
    // (right side, whose own direction is reversed): table values with the
    // sign bit set by an integer xor, no FP64 multiply
    const unsigned long long neg = right ? 0ull : 0x8000000000000000ull;
    auto sgn = [neg](double x) { return __longlong_as_double(__double_as_longlong(x) ^ neg); };
    const double2 p0 = *reinterpret_cast<const double2*>(m.etb + (3 * e + k) * 4);
    const double2 p1 = *reinterpret_cast<const double2*>(m.etb + (3 * e + k) * 4 + 2);
    const double s0 = sgn(m0);  // mode 1 is the constant phi_{e,1}
    const double b10 = sgn(right ? p1.x : p0.x), b11 = sgn(right ? p0.x : p1.x);
    const double b20 = sgn(right ? p1.y : p0.y), b21 = sgn(right ? p0.y : p1.y);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      r[f][0] += s0 * (F[f][0] + F[f][1]);
      r[f][1] += F[f][0] * b10 + F[f][1] * b11;
      r[f][2] += F[f][0] * b20 + F[f][1] * b21;
    }
  }
  // correction of the base modes from the volume terms of p >= 2 elements
  if (!stg.base_only && e >= rc_start) {
    const int64_t nrc = ne - rc_start, lr = e - rc_start;
    r[1][1] += rc[0 * nrc + lr];
    r[1][2] += rc[1 * nrc + lr];
    r[2][1] += rc[2 * nrc + lr];
    r[2][2] += rc[3 * nrc + lr];
  }
  const int K = m.p[e] == 0 ? 1 : 3;
  const double dt = stage_dt(stg, m.mem[e]), a = stg.a, bb = stg.b;
  const bool euler = a == 0.0 && bb == 1.0;  // the first stage: c + dt r
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int64_t ix = (f * 3 + q) * ne + e;
      double v = 0.0;
      if (q < K) {
        if (stg.rhs_only) v = r[f][q];
        else if (euler) v = c[f][q] + dt * r[f][q];
        else v = (a != 0.0 ? a * cbN[ix] : 0.0) + bb * (c[f][q] + dt * r[f][q]);
      }
      cbO[ix] = v;
      if (cbO32) cbO32[ix] = (float)v;
    }
  });
}

int launch_elem_base(cudaStream_t s, const DevMesh& m, const Groups& G, const Phys& ph, const Stage& stg,
                     const double* cbS, const double* cbN, double* cbO, float* cbO32, const double* ub, EdgeFlux fx,
                     const void* rc, unsigned* work) {
  if (m.ne == 0) return 0;
  const LaunchShape& L = launch_shape();
  const int nb = capped_blocks(m.ne, L.base_threads, L.base_bpsm);
  if (L.base_bpsm == 0 || L.base_bpsm >= 4)
    k_elem_base<4><<<nb, L.base_threads, 0, s>>>(m, ph, stg, cbS, cbN, cbO, cbO32, ub, fx.Fb, fx.Fbc,
                                                 (const double*)rc, G.start[2], base_chunk(L), work);
  else
    k_elem_base<3><<<nb, L.base_threads, 0, s>>>(m, ph, stg, cbS, cbN, cbO, cbO32, ub, fx.Fb, fx.Fbc,
                                                 (const double*)rc, G.start[2], base_chunk(L), work);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------------------
// p-adaptivity indicator (modal decay of xi, FP64 in every mode):
//   s_e = sum_{deg i = p_e} xi_i^2 / sum_{deg i >= 1} xi_i^2
// p_e + 1 if s_e > theta_up (p_e < p_max), p_e - 1 if s_e < theta_down
// (p_e > p_min).  The new orders are written in the caller's element order.
// ---------------------------------------------------------------------------
template <typename TC>
__global__ void k_indicator(DevMesh m, Groups G, const int32_t* __restrict__ perm, StateDev st, double up,
                            double down, int pmin, int pmax, int8_t* __restrict__ p_user) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int64_t ne = m.ne;
  const int p = m.p[e], K = Kof(p);
  double num = 0.0, den = 0.0;
  for (int i = 1; i < K && i < 3; ++i) {
    const double x = st.cb[i * ne + e];
    den += x * x;
    if (p == 1) num += x * x;
  }
  if (p >= 2) {
    const int64_t n = G.start[p + 1] - G.start[p], l = e - G.start[p];
    const TC* h = chp<TC>(st.ch[p]);
    for (int i = 3; i < K; ++i) {
      const double x = (double)h[(i - 3) * n + l];
      den += x * x;
      if (deg_of(i) == p) num += x * x;
    }
  }
  const double s = (p > 0 && den > 0.0) ? num / den : 0.0;
  int q = p;
  if (s > up && p < pmax) q = p + 1;
  else if (s < down && p > pmin) q = p - 1;
  p_user[perm[e]] = (int8_t)q;
}

int launch_indicator(cudaStream_t s, const DevMesh& m, const Groups& G, const int32_t* perm, int corr_fp32,
                     StateDev st, double up, double down, int pmin, int pmax, int8_t* p_user) {
  if (m.ne == 0) return 0;
  if (corr_fp32) k_indicator<float><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, perm, st, up, down, pmin, pmax, p_user);
  else k_indicator<double><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, perm, st, up, down, pmin, pmax, p_user);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------------------
// status: non-finite values in the state
// ---------------------------------------------------------------------------
template <typename TC>
__global__ void k_check(DevMesh m, Groups G, StateDev st, unsigned* status) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.ne) return;
  const int64_t ne = m.ne;
  bool bad = false;
  for (int i = 0; i < 9; ++i) bad |= !isfinite(st.cb[i * ne + e]);
  const int p = m.p[e];
  if (p >= 2) {
    const int K = Kof(p);
    const int64_t n = G.start[p + 1] - G.start[p], l = e - G.start[p];
    const TC* h = chp<TC>(st.ch[p]);
    for (int i = 0; i < 3 * (K - 3); ++i) bad |= !isfinite((double)h[i * n + l]);
  }
  if (bad) {
    atomicOr(status, (unsigned)ST_NONFINITE);
    atomicOr(m.mstatus + m.mem[e], (unsigned)ST_NONFINITE);
  }
}

int launch_check_state(cudaStream_t s, const DevMesh& m, const Groups& G, int corr_fp32, StateDev st,
                       unsigned* status) {
  if (m.ne == 0) return 0;
  if (corr_fp32) k_check<float><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, st, status);
  else k_check<double><<<nblocks(m.ne, 256), 256, 0, s>>>(m, G, st, status);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------------------
// deterministic reductions (fixed tree per block, blocks summed in order)
// ---------------------------------------------------------------------------
__device__ void block_sum_store(double v, double* partial) {
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* partial, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s;
  }
}

__global__ void k_mass(DevMesh m, const double* __restrict__ cb, double* partial) {
  double v = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.ne; e += (int64_t)gridDim.x * blockDim.x)
    v += m.geo[G_SQA * m.ne + e] * cb[e];
  block_sum_store(v, partial);
}

int launch_mass(cudaStream_t s, const DevMesh& m, const double* cb, double* partial, int nblk, double* out) {
  k_mass<<<nblk, 256, 0, s>>>(m, cb, partial);
  count_launch();
  k_sum_partials<<<1, 32, 0, s>>>(partial, nblk, out);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

template <typename TC>
__global__ void k_energy(DevMesh m, Groups G, Phys ph, StateDev c, VelDev u, double* partial) {
  double v = 0.0;
  const int64_t ne = m.ne;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = m.p[e], K = Kof(p);
    for (int i = 0; i < 3 && i < K; ++i) {
      const double x = c.cb[i * ne + e];
      v += 0.5 * ph.g * x * x + 0.5 * (c.cb[(3 + i) * ne + e] * u.ub[i * ne + e] + c.cb[(6 + i) * ne + e] * u.ub[(3 + i) * ne + e]);
    }
    if (p >= 2) {
      const int64_t n = G.start[p + 1] - G.start[p], l = e - G.start[p];
      const TC* h = chp<TC>(c.ch[p]);
      const TC* uh = chp<TC>(u.uh[p]);
      const int Kh = K - 3;
      for (int i = 0; i < Kh; ++i) {
        const double x = h[i * n + l];
        v += 0.5 * ph.g * x * x + 0.5 * ((double)h[(Kh + i) * n + l] * (double)uh[i * n + l] +
                                         (double)h[(2 * Kh + i) * n + l] * (double)uh[(Kh + i) * n + l]);
      }
    }
  }
  block_sum_store(v, partial);
}

int launch_energy(cudaStream_t s, const DevMesh& m, const Groups& G, int corr_fp32, const Phys& ph, StateDev c,
                  VelDev u, double* partial, int nblk, double* out) {
  if (corr_fp32) k_energy<float><<<nblk, 256, 0, s>>>(m, G, ph, c, u, partial);
  else k_energy<double><<<nblk, 256, 0, s>>>(m, G, ph, c, u, partial);
  count_launch();
  k_sum_partials<<<1, 32, 0, s>>>(partial, nblk, out);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

}  // namespace swedg
