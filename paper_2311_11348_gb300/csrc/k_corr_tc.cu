// FP32 correction with the momentum volume terms of Eq. (13) on the 5th-
// generation tensor cores (tcgen05, TF32 inputs, FP32 accumulation in TMEM).
//
// The correction kernels of k_corr_impl.cuh are instantiated once more here
// (namespace corrtc, FP32, CORR_TC): for the orders with K >= 10 modes
// k_elem_corr reads the volume terms of the U and V rows from a buffer
// instead of contracting them itself.  The buffer is written by k_vol_tc<K>.
//
// The contraction of one element (test modes q, coefficient rows i, j),
//   r_U[q] = (1/s) sum_{k,i,j} G_k[q][i][j] (U_i w^k_j + xi_i px^k_j)
//   r_V[q] = (1/s) sum_{k,i,j} G_k[q][i][j] (V_i w^k_j + xi_i py^k_j)
// with w = (uc, vc) the contravariant velocity coefficients (J^-1 u) and
// px^k = g J^-1_{k,x} pp, py^k = g J^-1_{k,y} pp, pp = xi/2, is done in
// two stages.  Stage one contracts over (k, j) for every (i, q) at once,
//   W[i][q]  = sum_{k,j} G_k[q][i][j] w^k_j
//   ZU[i][q] = sum_{k,j} G_k[q][i][j] px^k_j,   ZV[i][q] = ... py^k_j,
// which over a tile of 128 elements is three GEMMs with the SAME constant
// operand B[(i,q)][(k,j)] = G_k[q][i][j] (N = 16 K rows (i, q), q padded to
// 16; reduction 2 K columns (k, j)) and one per-element operand A each
// (rows = elements, the 2 K values w, px or py): M = 128, N = 160 or 240.
// Stage two, on the CUDA cores, contracts over i with the element's own
// coefficients: r_U[q] = (1/s) sum_i (U_i W[i][q] + xi_i ZU[i][q]) and
// r_V[q] = (1/s) sum_i (V_i W[i][q] + xi_i ZV[i][q]), each thread reading
// its element's row of the accumulators from TMEM.  The tensor cores carry
// 6 K^3 multiply-adds per element in large instructions (128 x 240 x 8), and
// the operands the threads form are 2 K values per GEMM, not K^2 products.
// B is zero for the base triples q, i, j < 3 (the FP64 base kernels own them)
// and for structural zeros.
//
// Precision: every FP32 operand x is split into two TF32 parts, x = h + t
// to within 2^-22 |x|, with h = tf32(x) and t = tf32(x - h) (tf32 = round to
// the nearest value with 10 mantissa bits), and each GEMM runs as the three
// products hh + ht + th into one FP32 accumulator.  The B parts come from the
// FP64 values of G.  The bottom term g xi h_b keeps only the products with a
// higher elevation mode (i >= 3; the correction edge kernel carries the rest
// as g h_b times the FP64 jump of the degree-1 elevation), which the GEMM's
// shared operand cannot single out: it is added on the CUDA cores after the
// GEMMs, g sum_{i >= 3, j < 3} xi_i h_b_j sum_k J^-1_k G_k[q][i][j].
//
// Schedule: one persistent CTA per SM (128 threads, thread t = element row t
// of the tile) loads both parts of B once (bulk TMA copies on an mbarrier),
// then per tile: the threads write the A operands (both parts) into shared
// memory; one thread issues the MMAs and commits them to an mbarrier; every
// thread reads its TMEM row and finishes stage two.  TMEM: 512 columns, one
// accumulator of N columns per GEMM; for K = 15 (3 x 240 > 512) the third
// GEMM runs in a second pass over the columns of the first.
//
// Shared-memory operand layout: K-major with the 128-byte swizzle.  A row is
// 32 floats = 128 bytes (the reduction padded to 32 with zeros); groups of 8
// rows are 1024 bytes apart (the descriptor's stride-dimension byte offset),
// and the 16-byte unit u of row r is stored at unit u ^ (r % 8): (row r,
// column c) at float offset
//   (r / 8) * 256 + (r % 8) * 32 + (((c / 4) ^ (r % 8)) * 4) + c % 4.
// An MMA step k of 8 columns starts 32 bytes further into the rows.
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

constexpr int TC_M = 128;     // elements per tile = MMA M
constexpr int TC_KD = 32;     // reduction columns of a row (2 K, padded)
constexpr int TC_COLS = 512;  // TMEM columns per CTA
constexpr int TC_PARTS = 2;   // TF32 parts of every operand: head, tail
constexpr int TC_ABUF = TC_M * TC_KD;  // floats of one part of one A operand
constexpr uint32_t TC_SPIN = 1u << 22;

// B rows (= MMA N) and reduction steps of 8 for K modes; GEMMs per TMEM pass
__host__ __device__ constexpr int tc_nb(int K) { return 16 * K; }
__host__ __device__ constexpr int tc_ksteps(int K) { return (2 * K + 7) / 8; }
__host__ __device__ constexpr int tc_pass_gemms(int K) { return 3 * tc_nb(K) <= TC_COLS ? 3 : 2; }
// floats of one part of the B image, of both parts, and the offset of K's image
__host__ __device__ constexpr int tc_bpart(int K) { return tc_nb(K) * TC_KD; }
__host__ __device__ constexpr int tc_bfloats(int K) { return TC_PARTS * tc_bpart(K); }
__host__ __device__ constexpr int tc_boff(int K) {
  return K == 6 ? 0 : K == 10 ? tc_bfloats(6) : tc_bfloats(6) + tc_bfloats(10);
}
constexpr int TC_BTOTAL = tc_bfloats(6) + tc_bfloats(10) + tc_bfloats(15);
// float offset of (row r, column c) in a K-major operand with the 128-byte swizzle
__host__ __device__ constexpr int tc_at(int r, int c) {
  return (r / 8) * 256 + (r % 8) * 32 + (((c / 4) ^ (r % 8)) * 4) + (c % 4);
}
// shared memory of k_vol_tc<K>: B (both parts), three A operands (both parts), barriers + TMEM slot
__host__ __device__ constexpr int tc_smem(int K) { return (tc_bfloats(K) + 3 * TC_PARTS * TC_ABUF) * 4 + 64; }

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
  std::fill(out, out + need, 0.0f);
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < K; ++q)
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
          if (!gnz(q, i, j) || base3(q, i, j)) continue;
          const int row = 16 * i + q, col = k * K + j;
          double rest = R.G[k][q][i][j];
          for (int part = 0; part < TC_PARTS; ++part) {
            const float v = tf32_round((float)rest);
            rest -= (double)v;
            out[part * tc_bpart(K) + tc_at(row, col)] = v;
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
// the 16-byte groups of one A row: values v[c] (c < 2K, zero beyond), both parts
template <int K>
__device__ __forceinline__ void write_a_row(float* aH, float* aT, int r, const float (&v)[TC_KD]) {
#pragma unroll
  for (int c4 = 0; c4 < tc_ksteps(K) * 2; ++c4) {  // the columns the MMA steps read
    float x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = v[4 * c4 + q];
    float4 h4, t4;
    split4(x, h4, t4);
    const int off = tc_at(r, 4 * c4);
    *reinterpret_cast<float4*>(aH + off) = h4;
    *reinterpret_cast<float4*>(aT + off) = t4;
  }
}

template <int K>
__global__ void __launch_bounds__(TC_M, 1) k_vol_tc(DevMesh m, int64_t g0, int64_t n, int64_t rc_off, int64_t nrc,
                                                     Phys ph, const float* __restrict__ cb,
                                                     const float* __restrict__ ch, const float* __restrict__ ub,
                                                     const float* __restrict__ uh, const float* __restrict__ bimg,
                                                     float* __restrict__ vol, unsigned* status) {
  constexpr int NB = tc_nb(K), KS = tc_ksteps(K), PG = tc_pass_gemms(K), BP = tc_bpart(K);
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  float* sB = reinterpret_cast<float*>(tc_smem_raw);  // [part][NB rows][32]
  float* sA = sB + TC_PARTS * BP;                      // [operand W, ZU, ZV][part][128 rows][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 3 * TC_PARTS * TC_ABUF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const int t = threadIdx.x, w = t >> 5;
  const uint32_t bfull = smem_u32(bars), mdone = smem_u32(bars + 1);
  if (t == 0) {
    mbar_init(bfull, 1);
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (t == 0) {  // both parts of B, once per CTA
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(bfull), "r"((uint32_t)(TC_PARTS * BP * 4))
                 : "memory");
#pragma unroll
    for (int part = 0; part < TC_PARTS; ++part)
      bulk_g2s(smem_u32(sB + part * BP), bimg + part * BP, (uint32_t)(BP * 4), bfull);
  }
  // the swizzle XOR acts on address bits 4-9: operands must start on 1024 bytes
  bool ok = (smem_u32(sA) & 1023u) == 0 && (smem_u32(sB) & 1023u) == 0;
  bool bready = false;
  uint32_t commits = 0;
  const uint32_t idesc = tc_idesc(TC_M, NB);
  const uint32_t lane_base = tmem + ((uint32_t)(32 * w) << 16);
  const float* geo = m.geo32;
  const int64_t ne = m.ne;
  const float g = (float)ph.g;

  // the MMAs of `ng` GEMMs, operand a0 + gi into TMEM columns col0 + gi * NB, then a commit
  auto issue = [&](int a0, int ng, uint32_t col0) {
    if (t == 0) {
      if (!bready) {
        ok &= mbar_wait(bfull, 0);
        bready = true;
      }
      tc_fence_after();
      const uint32_t b0 = smem_u32(sB), bpb = BP * 4;
      for (int gi = 0; gi < ng; ++gi) {
        const uint32_t a = smem_u32(sA + (a0 + gi) * TC_PARTS * TC_ABUF), apb = TC_ABUF * 4;
        const uint32_t d = tmem + col0 + (uint32_t)(gi * NB);
#pragma unroll
        for (int st = 0; st < KS; ++st) {  // K = 8 per MMA: 32 bytes further into the swizzled rows
          const uint32_t o = 32u * st;
          tc_mma(d, tc_desc(a + o), tc_desc(b0 + o), idesc, st > 0 ? 1u : 0u);  // h h
          tc_mma(d, tc_desc(a + o), tc_desc(b0 + bpb + o), idesc, 1u);           // h t
          tc_mma(d, tc_desc(a + apb + o), tc_desc(b0 + o), idesc, 1u);           // t h
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mdone)
                   : "memory");
    }
  };
  auto wait_mma = [&]() {
    const bool r = mbar_wait(mdone, commits & 1u);
    ++commits;
    ok &= r;
    tc_fence_after();
    return r;
  };

#pragma unroll 1
  for (int64_t tile = blockIdx.x; tile * TC_M < n; tile += gridDim.x) {
    const int64_t l = tile * TC_M + t;
    const bool live = l < n;
    const int64_t e = g0 + (live ? l : 0);
    float xi[K], U[K], V[K], pp[K];
    float J0 = 0.f, J1 = 0.f, J2 = 0.f, J3 = 0.f, rs = 0.f, hb[3] = {0.f, 0.f, 0.f};
    float aw[TC_KD], ax[TC_KD];
#pragma unroll
    for (int c = 0; c < TC_KD; ++c) aw[c] = ax[c] = 0.0f;
    if (live) {
      J0 = geo[G_JI0 * ne + e]; J1 = geo[G_JI1 * ne + e];
      J2 = geo[G_JI2 * ne + e]; J3 = geo[G_JI3 * ne + e];
      rs = geo[G_RS * ne + e];
      hb[0] = geo[G_HB0 * ne + e];
      hb[1] = geo[G_HB1 * ne + e];
      hb[2] = geo[G_HB2 * ne + e];
      float uu[K], vv[K];
      load_modes<K>(xi, cb, ne, e, ch, n, l, 0);
      load_modes<K>(U, cb, ne, e, ch, n, l, 1);
      load_modes<K>(V, cb, ne, e, ch, n, l, 2);
      load_modes<K>(uu, ub, ne, e, uh, n, l, 0);
      load_modes<K>(vv, ub, ne, e, uh, n, l, 1);
      sfor<0, K>([&](auto j) {
        aw[j] = J0 * uu[j] + J1 * vv[j];       // uc
        aw[K + j] = J2 * uu[j] + J3 * vv[j];   // vc
        pp[j] = 0.5f * xi[j];  // h_b stays out of the GEMM (see the epilogue)
        ax[j] = g * J0 * pp[j];                // px (U equation)
        ax[K + j] = g * J2 * pp[j];
      });
    } else {
      sfor<0, K>([&](auto j) { xi[j] = U[j] = V[j] = pp[j] = 0.0f; });
    }
    write_a_row<K>(sA, sA + TC_ABUF, t, aw);
    write_a_row<K>(sA + 2 * TC_ABUF, sA + 3 * TC_ABUF, t, ax);
    auto zv_row = [&](float (&ay)[TC_KD]) {
#pragma unroll
      for (int c = 0; c < TC_KD; ++c) ay[c] = 0.0f;
      sfor<0, K>([&](auto j) {
        ay[j] = g * J1 * pp[j];  // py (V equation)
        ay[K + j] = g * J3 * pp[j];
      });
    };
    if constexpr (PG == 3) {
      float ay[TC_KD];
      zv_row(ay);
      write_a_row<K>(sA + 4 * TC_ABUF, sA + 5 * TC_ABUF, t, ay);
    }
    // publish the rows to the tensor cores' (async) proxy; the previous tile's
    // TMEM reads are complete (tcgen05.wait::ld) before the barrier
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    issue(0, PG, 0u);
    wait_mma();
    // block-uniform: tcgen05.ld is a warp-wide instruction and the barriers below need every thread
    const bool got = __syncthreads_and(ok) != 0;
    if (!got) ok = false;
    float rU[16], rV[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) rU[q] = rV[q] = 0.0f;
    if (got) {
      sfor<0, K>([&](auto i) {
        float wv[16], zu[16];
        tmem_ld16(lane_base + (uint32_t)(16 * i), wv);
        tmem_ld16(lane_base + (uint32_t)(NB + 16 * i), zu);
        if constexpr (PG == 3) {
          float zv[16];
          tmem_ld16(lane_base + (uint32_t)(2 * NB + 16 * i), zv);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) rV[q] = fmaf(xi[i], zv[q], rV[q]);
        } else {
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          rU[q] = fmaf(U[i], wv[q], fmaf(xi[i], zu[q], rU[q]));
          rV[q] = fmaf(V[i], wv[q], rV[q]);
        }
      });
    }
    if constexpr (PG == 2) {  // ZV in a second pass over the first GEMM's columns
      if (!got) break;
      float ay[TC_KD];
      zv_row(ay);
      write_a_row<K>(sA, sA + TC_ABUF, t, ay);  // the W operand's MMAs are done
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      issue(0, 1, 0u);
      wait_mma();
      const bool got2 = __syncthreads_and(ok) != 0;
      if (!got2) ok = false;
      if (got2) {
        sfor<0, K>([&](auto i) {
          float zv[16];
          tmem_ld16(lane_base + (uint32_t)(16 * i), zv);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) rV[q] = fmaf(xi[i], zv[q], rV[q]);
        });
      }
    }
    // the bottom term's products with the higher elevation modes,
    // g sum_{i >= 3, j < 3} xi_i h_b_j sum_k J^-1_k G_k[q][i][j], in FP32 here
    float xh[K][3];
    sfor<3, K>([&](auto i) { sfor<0, 3>([&](auto j) { xh[i][j] = xi[i] * hb[j]; }); });
    sfor<1, K>([&](auto Q) {
      float ex = 0.f, ey = 0.f;
      sfor<3, K>([&](auto i) {
        sfor<0, 3>([&](auto j) {
          if constexpr (gnz(Q, i, j)) {
            ex = fmaf(xh[i][j], cG[0][Q][pk(i, j)], ex);
            ey = fmaf(xh[i][j], cG[1][Q][pk(i, j)], ey);
          }
        });
      });
      rU[Q] = fmaf(g, J0 * ex + J2 * ey, rU[Q]);
      rV[Q] = fmaf(g, J1 * ex + J3 * ey, rV[Q]);
    });
    if (live && ok) {
#pragma unroll
      for (int q = 1; q < K; ++q) {
        vol[q * nrc + rc_off + l] = rs * rU[q];
        vol[(16 + q) * nrc + rc_off + l] = rs * rV[q];
      }
    }
    tc_fence_before();
    // the next tile rewrites A and the accumulators; a failed wait anywhere ends the loop for all
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
  }
  if (!ok && t == 0) atomicOr(status, (unsigned)ST_TIMEOUT);
  // a commit still in flight (a wait that gave up) completes before TMEM is freed
  if (!ok && commits > 0) mbar_wait(mdone, (commits - 1) & 1u);
  if (!bready && t == 0) mbar_wait(bfull, 0);  // the B copies land before the CTA exits
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
  }
}

static_assert(tc_smem(15) <= 227 * 1024 && tc_smem(10) <= 227 * 1024, "shared memory of one CTA");
static_assert(tc_nb(15) <= 256 && tc_nb(15) % 16 == 0 && tc_nb(10) % 16 == 0, "MMA N");
static_assert(tc_pass_gemms(10) * tc_nb(10) <= TC_COLS && 2 * tc_nb(15) <= TC_COLS, "TMEM columns");

static int g_nsm_tc = 152;

template <int K>
static int vol_group(cudaStream_t st, const DevMesh& m, const Groups& G, int p, const Phys& ph, StateDev c, VelDev u,
                     float* vol, unsigned* status, const float* bimg) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  const int64_t nrc = G.start[5] - G.start[2], rc_off = g0 - G.start[2];
  const int64_t tiles = (n + TC_M - 1) / TC_M;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, g_nsm_tc);
  k_vol_tc<K><<<grid, TC_M, tc_smem(K), st>>>(m, g0, n, rc_off, nrc, ph, c.cb32, (const float*)c.ch[p], u.ub32,
                                             (const float*)u.uh[p], bimg + tc_boff(K), vol, status);
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
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(10)));
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<15>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(15)));
  int nsm = 0;
  SWE_CUDA_OK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (nsm > 0) g_nsm_tc = nsm;
  return 0;
}

}  // namespace corrtc
}  // namespace swedg
