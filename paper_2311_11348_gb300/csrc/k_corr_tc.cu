// FP32 correction with the momentum volume terms of Eq. (13) on the 5th-
// generation tensor cores (tcgen05, TF32 inputs, FP32 accumulation in TMEM).
//
// The correction kernels of k_corr_impl.cuh are instantiated once more here
// (namespace corrtc, FP32, CORR_TC): for the orders with K >= 10 modes
// k_elem_corr reads the volume terms of the U and V rows from a buffer
// instead of contracting them itself.  The buffer is written by k_vol_tc<K>,
// one CTA per 128 elements of one order group, as three GEMMs over the
// element tile (rows = elements):
//
//   D_U[e][q] = sum_{k,i,j} U_i w^k_j  G_k[q][i][j]      w^x = uc, w^y = vc
//   D_V[e][q] = sum_{k,i,j} V_i w^k_j  G_k[q][i][j]
//   D_P[e][(k,q)] = sum_{i,j} xi_i pp_j G_k[q][i][j]     pp = xi/2 + h_b
//
// (uc, vc: the contravariant velocity coefficients J^-1 u; pp without h_b's
// mean mode, which the epilogue adds: see there).  The reduction index runs
// over five "kinds" of coefficient products, (U, uc), (U, vc), (V, uc),
// (V, vc), (xi, pp), each a K x 16 block (i < K, j < 16, zero for j >= K);
// the B operands are the matching blocks of G (zero for the base triples
// q, i, j < 3, which the FP64 base kernels own, and for structural zeros).
// The epilogue forms, as the CUDA-core contraction does,
//   r_U[q] = (1/s) (D_U[q] + g (J00 D_P[x^,q] + J10 D_P[y^,q]))
//   r_V[q] = (1/s) (D_V[q] + g (J01 D_P[x^,q] + J11 D_P[y^,q])).
//
// Precision: every FP32 operand x is split into two TF32 parts, x = h + t
// to within 2^-22 |x|, with h = tf32(x) and t = tf32(x - h) (tf32 = round to
// the nearest value with 10 mantissa bits), and each GEMM runs as the three
// products hh + ht + th with FP32 accumulation.  The B operands (reference
// tensors) are split the same way from their FP64 values.  The mean depth
// (kilometres, against metres of elevation) would be the largest term of the
// pressure products; it enters only through hb0 * sum_i xi_i G_k[q][i][0],
// which the CUDA cores add in the epilogue.  With that, one right-hand side
// of this mode matches the FP64 oracle as closely as the FP32 CUDA-core
// contraction does (measured 0.5-1.2e-6 relative L2 for both).
//
// Pipeline (one CTA = 128 threads = 4 warps; thread t owns element row t):
// the reduction is cut into chunks of 32 columns (two rows i of one kind).
// A two-stage shared-memory ring holds the A chunks, formed by all threads
// from registers and a per-thread coefficient table in shared memory; each
// thread signals its rows of a chunk on the stage's "afull" mbarrier (128
// arrivals, no block barrier, so the other warps run a chunk ahead of thread
// 0).  A three-stage ring holds the B chunks, each brought by one bulk TMA
// copy per operand part (cp.async.bulk, complete_tx on the stage's "full"
// mbarrier) one chunk ahead of its use.  Thread 0 waits for both, issues the
// twelve MMAs of the chunk (four K = 8 steps x three products, the three
// products into three TMEM accumulator sets: independent MMA chains) and
// commits them to the A stage's "empty" mbarrier.  The chunk loop is a
// runtime loop (a fully unrolled one did not fit the instruction cache).
// TMEM: 256 columns per CTA, three sets of 64 (D_U 0..15, D_V 16..31, D_P
// 32..63), summed and read back with tcgen05.ld in the epilogue.
//
// Shared-memory operand layout: K-major with the 128-byte swizzle.  A row of
// a chunk is 32 floats = 128 bytes; rows are 128 bytes apart, groups of 8 rows
// 1024 bytes apart (the descriptor's stride-dimension byte offset), and the
// 16-byte unit u of row r is stored at unit u ^ (r % 8): (row r, column c) at
// float offset
//   (r / 8) * 256 + (r % 8) * 32 + (((c / 4) ^ (r % 8)) * 4) + c % 4
// (chunks start on 1024-byte boundaries, so the XOR matches the address bits
// the tensor cores swizzle with).  An MMA step k of 8 columns starts 32 bytes
// further into the rows.  The swizzle spreads a core matrix's rows over all
// banks; the unswizzled layout measured ~5000 cycles per 32-column chunk.
//
// Every mbarrier wait is bounded; a wait that runs out sets ST_TIMEOUT in the
// status word, skips the result and still frees the CTA's TMEM.
#include <algorithm>
#include <cstring>

#define CORR_T float
#define CORR_NS corrtc
#define CORR_TC 1
#include "k_corr_impl.cuh"

namespace swedg {
namespace corrtc {

constexpr int TC_M = 128;    // elements per CTA = MMA M
constexpr int TC_NS = 16;    // N of the U / V GEMMs (q = 0..15)
constexpr int TC_NP = 32;    // N of the P GEMM (x^ q, then y^ q)
constexpr int TC_W = 16;     // columns per coefficient row i (j < 16)
constexpr int TC_ACC = 64;   // TMEM columns of one accumulator set (D_U, D_V, D_P)
constexpr int TC_COLS = 256; // TMEM columns per CTA: hh, ht, th accumulator sets (a power of 2)
constexpr int TC_BST = 3;    // stages of the B ring (a chunk's B is copied one chunk ahead)
constexpr int TC_PARTS = 2;  // TF32 parts of every operand: head, tail
constexpr int TC_ABUF = TC_M * 32;   // floats of one part of one A chunk
constexpr int TC_BSLOT = TC_NP * 32; // floats of one part of one B chunk (the larger, P)
constexpr uint32_t TC_SPIN = 1u << 22;

// Chunk c covers rows 2 (c / 5) and 2 (c / 5) + 1 of kind tc_kind(c): the kinds
// alternate (U,uc) (V,uc) (U,vc) (V,vc) (xi,pp) so that consecutive chunks
// accumulate into different TMEM sets (D_U, D_V, D_U, D_V, D_P) and their MMA
// chains overlap; the first chunk of each set is in the first round.
__host__ __device__ constexpr int tc_kind(int c) { return c % 5 == 1 ? 2 : c % 5 == 2 ? 1 : c % 5; }
// chunks per kind (two rows i per chunk) and in all
__host__ __device__ constexpr int tc_cpk(int K) { return (K + 1) / 2; }
__host__ __device__ constexpr int tc_nchunks(int K) { return 5 * tc_cpk(K); }
// floats of one part of the B image: the x^ and y^ chunks of the U / V GEMMs, then the P chunks
__host__ __device__ constexpr int tc_bpart(int K) { return tc_cpk(K) * (2 * TC_NS * 32 + TC_NP * 32); }
__host__ __device__ constexpr int tc_bfloats(int K) { return TC_PARTS * tc_bpart(K); }
__host__ __device__ constexpr int tc_boff(int K) {
  return K == 6 ? 0 : K == 10 ? tc_bfloats(6) : tc_bfloats(6) + tc_bfloats(10);
}
constexpr int TC_BTOTAL = tc_bfloats(6) + tc_bfloats(10) + tc_bfloats(15);
// float offset of (row r, column c) in a chunk of 32 columns
__host__ __device__ constexpr int tc_at(int r, int c) {
  return (r / 8) * 256 + (r % 8) * 32 + (((c / 4) ^ (r % 8)) * 4) + (c % 4);
}
// shared memory of k_vol_tc: A ring, B ring, per-thread U, V, xi rows, barriers + TMEM slot
constexpr int TC_SMEM = (2 * TC_PARTS * TC_ABUF + TC_BST * TC_PARTS * TC_BSLOT + 3 * TC_W * TC_M) * 4 + 96;
static_assert((TC_BST + 4) * 8 + 4 <= 96, "barriers and TMEM slot");

__device__ __align__(128) float gTcB[TC_BTOTAL];
static const float* g_tcb[64];  // device address of gTcB per device ordinal

// round to the nearest value with a 10-bit mantissa (ties away from zero)
static inline float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xffffe000u;
  float h;
  std::memcpy(&h, &u, 4);
  return h;
}

int64_t tc_operand_image(int K, float* out, int64_t cap) {
  if (K != 6 && K != 10 && K != 15) return -1;
  const int64_t need = tc_bfloats(K);
  if (!out) return need;
  if (cap < need) return -1;
  const RefTables& R = tables();
  const int CPK = tc_cpk(K);
  std::fill(out, out + need, 0.0f);
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < K; ++q)
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
          if (!gnz(q, i, j) || base3(q, i, j)) continue;
          const int c = i / 2, col = (i % 2) * TC_W + j;
          double rest = R.G[k][q][i][j];
          for (int part = 0; part < TC_PARTS; ++part) {
            const float v = tf32_round((float)rest);
            rest -= (double)v;
            float* base = out + part * tc_bpart(K);
            base[(k * CPK + c) * (TC_NS * 32) + tc_at(q, col)] = v;                        // U / V GEMMs
            base[2 * CPK * (TC_NS * 32) + c * (TC_NP * 32) + tc_at(16 * k + q, col)] = v;  // P GEMM
          }
        }
  return need;
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle (layout type 2),
// SBO 1024 B between groups of 8 rows; LBO is not used by swizzled K-major
// layouts whose K step fits in the 128-byte row (encoded as 1)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  for (uint32_t it = 0; it < TC_SPIN; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// one bulk TMA copy global -> shared, completing on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_rn(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u); }

// x = h + t to within 2^-22 |x|, both parts TF32 values
__device__ __forceinline__ void split4(const float (&v)[4], float4& h4, float4& t4) {
  float h[4], t[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = tf32_rn(v[i]);
    t[i] = tf32_rn(v[i] - h[i]);
  }
  h4 = make_float4(h[0], h[1], h[2], h[3]);
  t4 = make_float4(t[0], t[1], t[2], t[3]);
}

// ------------------------------------------------------------ kernel
template <int K>
__global__ void __launch_bounds__(TC_M) k_vol_tc(DevMesh m, int64_t g0, int64_t n, int64_t rc_off, int64_t nrc,
                                                  Phys ph, const float* __restrict__ cb, const float* __restrict__ ch,
                                                  const float* __restrict__ ub, const float* __restrict__ uh,
                                                  const float* __restrict__ bimg, float* __restrict__ vol,
                                                  unsigned* status) {
  constexpr int CPK = tc_cpk(K), NC = tc_nchunks(K), BP = tc_bpart(K);
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  float* sA = reinterpret_cast<float*>(tc_smem_raw);  // [stage][part][TC_ABUF]
  float* sB = sA + 2 * TC_PARTS * TC_ABUF;             // [B stage][part][TC_BSLOT]
  float* sv = sB + TC_BST * TC_PARTS * TC_BSLOT;       // [U, V, xi][i < 16][thread]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sv + 3 * TC_W * TC_M);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + TC_BST + 4);
  const int t = threadIdx.x, w = t >> 5;
  // mbarriers: per A stage afull (A chunk written: all 128 threads) and empty (the chunk's MMAs
  // done: tcgen05.commit); per B stage full (B chunk landed: TMA bytes)
  const uint32_t bar0 = smem_u32(bars);
  auto empty = [&](int b) { return bar0 + 8u * b; };
  auto afull = [&](int b) { return bar0 + 16u + 8u * b; };
  auto full = [&](int bs) { return bar0 + 32u + 8u * bs; };

  if (t == 0) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      mbar_init(empty(b), 1);
      mbar_init(afull(b), TC_M);
    }
#pragma unroll
    for (int bs = 0; bs < TC_BST; ++bs) mbar_init(full(bs), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // this thread's element: U, V, xi rows to shared memory (read back by row
  // index), the velocity products' w rows in registers
  const int64_t l = (int64_t)blockIdx.x * TC_M + t;
  const bool live = l < n;
  const int64_t e = g0 + (live ? l : 0), ne = m.ne;
  const float* geo = m.geo32;
  float xi[K], uc[TC_W], vc[TC_W], pp[TC_W];
  float J0 = 0.f, J1 = 0.f, J2 = 0.f, J3 = 0.f, rs = 0.f, hb0 = 0.f;
#pragma unroll
  for (int j = 0; j < TC_W; ++j) uc[j] = vc[j] = pp[j] = 0.0f;
  {
    float U[K], V[K];
    if (live) {
      J0 = geo[G_JI0 * ne + e]; J1 = geo[G_JI1 * ne + e];
      J2 = geo[G_JI2 * ne + e]; J3 = geo[G_JI3 * ne + e];
      rs = geo[G_RS * ne + e];
      hb0 = geo[G_HB0 * ne + e];
      float uu[K], vv[K];
      load_modes<K>(xi, cb, ne, e, ch, n, l, 0);
      load_modes<K>(U, cb, ne, e, ch, n, l, 1);
      load_modes<K>(V, cb, ne, e, ch, n, l, 2);
      load_modes<K>(uu, ub, ne, e, uh, n, l, 0);
      load_modes<K>(vv, ub, ne, e, uh, n, l, 1);
      sfor<0, K>([&](auto j) {
        uc[j] = J0 * uu[j] + J1 * vv[j];
        vc[j] = J2 * uu[j] + J3 * vv[j];
        // h_b's mean mode stays out of the GEMM (see the epilogue)
        if constexpr (j == 1 || j == 2) pp[j] = 0.5f * xi[j] + geo[(G_HB0 + j) * ne + e];
        else pp[j] = 0.5f * xi[j];
      });
    } else {
      sfor<0, K>([&](auto j) { xi[j] = U[j] = V[j] = 0.0f; });
    }
    sfor<0, TC_W>([&](auto i) {
      if constexpr (i < K) {
        sv[(0 * TC_W + i) * TC_M + t] = U[i];
        sv[(1 * TC_W + i) * TC_M + t] = V[i];
        sv[(2 * TC_W + i) * TC_M + t] = xi[i];
      } else {
        sv[(0 * TC_W + i) * TC_M + t] = 0.0f;
        sv[(1 * TC_W + i) * TC_M + t] = 0.0f;
        sv[(2 * TC_W + i) * TC_M + t] = 0.0f;
      }
    });
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // B chunk of chunk cc into B stage cc % TC_BST: one bulk copy per part (thread 0)
  auto issue_b = [&](int cc) {
    const int kind = tc_kind(cc), cl = cc / 5, bs = cc % TC_BST;
    const bool P = kind == 4;
    const int off = P ? 2 * CPK * (TC_NS * 32) + cl * (TC_NP * 32) : ((kind & 1) * CPK + cl) * (TC_NS * 32);
    const uint32_t bytes = (P ? TC_NP : TC_NS) * 32 * 4;
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(full(bs)), "r"(TC_PARTS * bytes)
                 : "memory");
#pragma unroll
    for (int part = 0; part < TC_PARTS; ++part)
      bulk_g2s(smem_u32(sB + (bs * TC_PARTS + part) * TC_BSLOT), bimg + part * BP + off, bytes, full(bs));
  };
  if (t == 0) issue_b(0);

  // the swizzle XOR acts on address bits 4-9: every chunk must start on 1024 bytes
  bool ok = (smem_u32(sA) & 1023u) == 0 && (smem_u32(sB) & 1023u) == 0;
  float wv[TC_W];
#pragma unroll 1
  for (int c = 0; c < NC; ++c) {
    const int b = c & 1, use = c >> 1;
    const int kind = tc_kind(c), cl = c / 5;  // kinds: (U,uc) (U,vc) (V,uc) (V,vc) (xi,pp)
    if (c >= 2) ok &= mbar_wait(empty(b), (use - 1) & 1);  // MMAs of chunk c - 2 done: stage b is free
    // B of the next chunk, one chunk ahead: its B stage was last read by chunk c - 2, done above
    if (t == 0 && c + 1 < NC) issue_b(c + 1);
    {  // the w row of this kind
      const int wk = kind == 4 ? 2 : (kind & 1);
#pragma unroll
      for (int j = 0; j < TC_W; ++j) wv[j] = wk == 0 ? uc[j] : wk == 1 ? vc[j] : pp[j];
    }
    const int sk = kind == 4 ? 2 : (kind >> 1);  // U, V or xi
    float* aH = sA + (b * TC_PARTS) * TC_ABUF;
    float* aT = aH + TC_ABUF;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const float si = sv[(sk * TC_W + 2 * cl + rr) * TC_M + t];
#pragma unroll
      for (int j4 = 0; j4 < TC_W / 4; ++j4) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = si * wv[4 * j4 + q];
        float4 h4, t4;
        split4(v, h4, t4);
        const int off = tc_at(t, rr * TC_W + 4 * j4);
        *reinterpret_cast<float4*>(aH + off) = h4;
        *reinterpret_cast<float4*>(aT + off) = t4;
      }
    }
    // publish this thread's rows of the A chunk to the tensor cores' (async) proxy;
    // no block barrier: the other warps run on to the next chunk while thread 0 issues
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    {
      uint64_t state;
      asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(afull(b)) : "memory");
    }
    if (t == 0) {
      const int bs = c % TC_BST;
      ok &= mbar_wait(afull(b), use & 1);               // every row of the A chunk written
      ok &= mbar_wait(full(bs), (c / TC_BST) & 1);      // B chunk landed
      tc_fence_after();
      const bool P = kind == 4;
      const uint32_t idesc = P ? tc_idesc(TC_M, TC_NP) : tc_idesc(TC_M, TC_NS);
      const uint32_t d = tmem + (P ? 32u : (kind >> 1) ? 16u : 0u);
      const uint32_t acc0 = (cl == 0 && (kind & 1) == 0) ? 0u : 1u;  // first chunk of D_U, D_V or D_P
      const uint32_t a0 = smem_u32(aH), b0 = smem_u32(sB + (bs * TC_PARTS) * TC_BSLOT);
      const uint32_t ap = TC_ABUF * 4, bp = TC_BSLOT * 4;  // bytes between the parts
      // the three products accumulate in three TMEM sets (independent MMA chains), summed in the epilogue
#pragma unroll
      for (int s = 0; s < 4; ++s) {  // K = 8 per MMA: 32 bytes further into the swizzled rows
        const uint32_t o = 32u * s, acc = s == 0 ? acc0 : 1u;
        tc_mma(d, tc_desc(a0 + o), tc_desc(b0 + o), idesc, acc);                          // h h
        tc_mma(d + TC_ACC, tc_desc(a0 + o), tc_desc(b0 + bp + o), idesc, acc);            // h t
        tc_mma(d + 2 * TC_ACC, tc_desc(a0 + ap + o), tc_desc(b0 + o), idesc, acc);       // t h
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(empty(b))
                   : "memory");
    }
  }

  // the last commit covers every MMA of the tile
  constexpr int CL = NC - 1;
  bool done = mbar_wait(empty(CL & 1), (CL >> 1) & 1);
  ok &= done;
  __syncwarp();
  tc_fence_after();
  float dU[16], dV[16], dPx[16], dPy[16];
  const uint32_t lane_base = tmem + ((uint32_t)(32 * w) << 16);
  {
    float a[16], b2[16];
    auto ld_sum = [&](uint32_t col, float (&out)[16]) {  // hh + (ht + th)
      tmem_ld16(lane_base + col, out);
      tmem_ld16(lane_base + TC_ACC + col, a);
      tmem_ld16(lane_base + 2 * TC_ACC + col, b2);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) out[i] += a[i] + b2[i];
    };
    ld_sum(0, dU);
    ld_sum(16, dV);
    ld_sum(32, dPx);
    ld_sum(48, dPy);
  }
  // the pressure products' mean-depth part, hb0 * sum_i xi_i G_k[q][i][0], in FP32 here
  sfor<1, K>([&](auto Q) {
    float ex = 0.f, ey = 0.f;
    sfor<0, K>([&](auto i) {
      if constexpr (gnz(Q, i, 0) && !base3(Q, i, 0)) {
        ex = fmaf(xi[i], cG[0][Q][pk(i, 0)], ex);
        ey = fmaf(xi[i], cG[1][Q][pk(i, 0)], ey);
      }
    });
    dPx[Q] = fmaf(hb0, ex, dPx[Q]);
    dPy[Q] = fmaf(hb0, ey, dPy[Q]);
  });
  if (live && ok) {
    const float g = (float)ph.g;
#pragma unroll
    for (int q = 1; q < K; ++q) {
      vol[q * nrc + rc_off + l] = rs * (dU[q] + g * (J0 * dPx[q] + J2 * dPy[q]));
      vol[(16 + q) * nrc + rc_off + l] = rs * (dV[q] + g * (J1 * dPx[q] + J3 * dPy[q]));
    }
  }
  if (!ok) atomicOr(status, (unsigned)ST_TIMEOUT);
  if (!done) mbar_wait(empty(CL & 1), (CL >> 1) & 1);  // bounded second wait before TMEM is freed
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
  }
}

static_assert(TC_SMEM <= 113 * 1024, "two CTAs of k_vol_tc per SM");
static_assert(TC_NS * 32 % 256 == 0 && TC_NP * 32 % 256 == 0, "whole row groups per chunk");

template <int K>
static int vol_group(cudaStream_t st, const DevMesh& m, const Groups& G, int p, const Phys& ph, StateDev c, VelDev u,
                     float* vol, unsigned* status, const float* bimg) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  const int64_t nrc = G.start[5] - G.start[2], rc_off = g0 - G.start[2];
  k_vol_tc<K><<<(unsigned)((n + TC_M - 1) / TC_M), TC_M, TC_SMEM, st>>>(
      m, g0, n, rc_off, nrc, ph, c.cb32, (const float*)c.ch[p], u.ub32, (const float*)u.uh[p], bimg + tc_boff(K),
      vol, status);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_vol_tc(cudaStream_t st, const DevMesh& m, const Groups& G, const Phys& ph, StateDev c, VelDev u,
                  float* vol, unsigned* status) {
  int dev = 0;
  SWE_CUDA_OK(cudaGetDevice(&dev));
  const float* bimg = (dev >= 0 && dev < 64) ? g_tcb[dev] : nullptr;
  if (!bimg) return -1;
  static_assert(!tc_vol(6) && tc_vol(10) && tc_vol(15), "orders on the tensor cores");
  int r = vol_group<10>(st, m, G, 3, ph, c, u, vol, status, bimg);
  if (!r) r = vol_group<15>(st, m, G, 4, ph, c, u, vol, status, bimg);
  return r;
}

// Self-test of the bounded waits: an mbarrier that nothing arrives on, waited
// for `spins` times; the wait runs out, the kernel sets ST_TIMEOUT and returns.
__global__ void k_wait_selftest(int64_t spins, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = false;
    for (int64_t it = 0; it < spins && !ok; ++it) {
      uint32_t r;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(r)
          : "r"(a), "r"(0u)
          : "memory");
      ok = r != 0;
    }
    if (!ok) atomicOr(status, (unsigned)ST_TIMEOUT);
  }
}

int launch_wait_selftest(cudaStream_t st, int64_t spins, unsigned* status) {
  k_wait_selftest<<<1, 32, 0, st>>>(spins, status);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

// B images and kernel attributes of the current device (once per context creation)
int upload_tc_tables() {
  static float img[TC_BTOTAL];
  tc_operand_image(6, img + tc_boff(6), tc_bfloats(6));
  tc_operand_image(10, img + tc_boff(10), tc_bfloats(10));
  tc_operand_image(15, img + tc_boff(15), tc_bfloats(15));
  SWE_CUDA_OK(cudaMemcpyToSymbol(gTcB, img, sizeof img));
  int dev = 0;
  SWE_CUDA_OK(cudaGetDevice(&dev));
  void* a = nullptr;
  SWE_CUDA_OK(cudaGetSymbolAddress(&a, gTcB));
  if (dev >= 0 && dev < 64) g_tcb[dev] = (const float*)a;
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<15>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
  return 0;
}

}  // namespace corrtc
}  // namespace swedg
