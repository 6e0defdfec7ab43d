// FP32 correction with the momentum volume terms of Eq. (13) on the 5th-
// generation tensor cores (tcgen05, TF32 inputs, FP32 accumulation in TMEM).
//
// The correction kernels of k_corr_impl.cuh are instantiated once more here
// (namespace corrtc, FP32, CORR_TC): k_elem_corr reads the volume terms of
// the U and V rows from a buffer instead of contracting them itself.  The
// buffer is written by k_vol_tc<K>, one CTA per 128 elements of one order
// group, as three GEMMs over the element tile:
//
//   D_U[e][q] = sum_r A_U[e][r] B_S[q][r]      r = (k, i <= j), k in {x^, y^}
//   D_V[e][q] = sum_r A_V[e][r] B_S[q][r]
//   D_P[e][n] = sum_r A_P[e][r] B_P[n][r]      r = (i <= j), n = (k, q)
//
// with the symmetrised products of the element's coefficients (G_k[q][i][j]
// is symmetric in i, j)
//   A_U[e][(k,ij)] = U_i w^k_j + U_j w^k_i   (U_i w^k_i when i = j), w^x = uc, w^y = vc
//   A_P[e][ij]     = xi_i pp_j + xi_j pp_i   (xi_i pp_i when i = j),  pp = xi/2 + h_b
//                    (without h_b's mean mode, which the epilogue adds: see there)
// and the reference tensors B_S[q][(k,ij)] = B_P[(k,q)][ij] = G_k[q][i][j]
// (zero for the base triples q, i, j < 3, which the FP64 base kernels own).
// The epilogue forms, as in the CUDA-core contraction,
//   r_U[q] = (1/s) (D_U[q] + g (J00 D_P[x^,q] + J10 D_P[y^,q]))
//   r_V[q] = (1/s) (D_V[q] + g (J01 D_P[x^,q] + J11 D_P[y^,q])).
//
// Precision: every FP32 operand x is split into two TF32 parts, x = h + t
// to within 2^-22 |x|, with h = tf32(x) and t = tf32(x - h) (tf32 = round to
// the nearest value with 10 mantissa bits), and each GEMM runs as the three
// products hh + ht + th with FP32 accumulation; the omitted tt and the
// residuals are below 2^-22 of the product.  The B operands (reference
// tensors) are split the same way from their FP64 values.  Measured against
// the FP64 oracle, one right-hand side of this mode is within 1.5-3e-6
// relative L2 where the FP32 CUDA-core contraction is within 0.5-1.4e-6; an
// exact three-part split with six products measured the same, so the
// difference comes from the tensor cores' FP32 accumulation, not from the
// operand split.
//
// Data movement: the B images (constant per K, built on the host in the
// tensor cores' canonical K-major layout) are staged into shared memory by
// one bulk TMA copy (cp.async.bulk, completion on an mbarrier).  The A
// products are formed by the 128 threads (thread = element row) 32 reduction
// columns at a time into a double-buffered shared-memory ring; one thread
// issues the MMAs of a chunk and commits them to the buffer's mbarrier, so
// forming chunk c + 1 overlaps the MMAs of chunk c.  Accumulators: 64 TMEM
// columns (D_U 0..15, D_V 16..31, D_P 32..63), read back with tcgen05.ld.
//
// Shared-memory operand layout (no swizzle, K-major): 8 x 4 "core matrices"
// of 8 rows x 16 bytes, row r / column k of a 32-column chunk at float offset
//   (r / 8) * 256 + (k / 4) * 32 + (r % 8) * 4 + (k % 4)
// i.e. leading-dimension byte offset 128 (next core matrix along k) and
// stride-dimension byte offset 1024 (next group of 8 rows).
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

constexpr int TC_M = 128;   // elements per CTA = MMA M
constexpr int TC_NS = 16;   // N of the U / V GEMMs (q = 0..15)
constexpr int TC_NP = 32;   // N of the P GEMM (x^ q, then y^ q)
constexpr int TC_COLS = 64; // TMEM columns per CTA
constexpr uint32_t TC_SPIN = 1u << 22;

__host__ __device__ constexpr int tc_P(int K) { return K * (K + 1) / 2; }
__host__ __device__ constexpr int tc_RS(int K) { return (2 * tc_P(K) + 31) / 32 * 32; }
__host__ __device__ constexpr int tc_RP(int K) { return (tc_P(K) + 31) / 32 * 32; }
constexpr int TC_PARTS = 2;  // TF32 parts of every operand: head, tail
// floats of the B image of K modes: S head, tail, then P head, tail
__host__ __device__ constexpr int tc_bfloats(int K) { return TC_PARTS * (TC_NS * tc_RS(K) + TC_NP * tc_RP(K)); }
// A buffers in the ring
__host__ __device__ constexpr int tc_nbuf(int K) { return 2; }
__host__ __device__ constexpr int tc_boff(int K) {
  return K == 6 ? 0 : K == 10 ? tc_bfloats(6) : tc_bfloats(6) + tc_bfloats(10);
}
constexpr int TC_BTOTAL = tc_bfloats(6) + tc_bfloats(10) + tc_bfloats(15);
// float offset of (row r, reduction column k) in an operand of R rows
__host__ __device__ constexpr int tc_at(int R, int r, int k) {
  return (k / 32) * (R * 32) + (r / 8) * 256 + ((k % 32) / 4) * 32 + (r % 8) * 4 + (k % 4);
}
// shared-memory bytes of k_vol_tc<K>: B image, the A buffers (two parts each), barriers, TMEM slot
__host__ __device__ constexpr int tc_smem(int K) { return tc_bfloats(K) * 4 + tc_nbuf(K) * TC_PARTS * TC_M * 32 * 4 + 64; }
// pair index (i <= j) -> j
__host__ __device__ constexpr int pair_j(int pr) {
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= pr) ++j;
  return j;
}

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
  const int P = tc_P(K), RS = tc_RS(K), RP = tc_RP(K);
  float* sp[TC_PARTS];
  float* pp[TC_PARTS];
  for (int k = 0; k < TC_PARTS; ++k) {
    sp[k] = out + k * TC_NS * RS;
    pp[k] = out + TC_PARTS * TC_NS * RS + k * TC_NP * RP;
  }
  std::fill(out, out + need, 0.0f);
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < K; ++q)
      for (int j = 0; j < K; ++j)
        for (int i = 0; i <= j; ++i) {
          if (!gnz(q, i, j) || base3(q, i, j)) continue;
          double rest = R.G[k][q][i][j];
          const int pr = pk(i, j);
          for (int part = 0; part < TC_PARTS; ++part) {
            const float v = tf32_round((float)rest);
            rest -= (double)v;
            sp[part][tc_at(TC_NS, q, k * P + pr)] = v;
            pp[part][tc_at(TC_NP, k * 16 + q, pr)] = v;
          }
        }
  return need;
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B, SBO 1024 B
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46);
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

// ------------------------------------------------------------ A products
// value of reduction column k (0..31) of chunk C for this thread's element
template <int K, int C, int k>
__device__ __forceinline__ float tc_value(const float (&xi)[K], const float (&U)[K], const float (&V)[K],
                                          const float (&uc)[K], const float (&vc)[K], const float (&pp)[K]) {
  constexpr int P = tc_P(K), nS = tc_RS(K) / 32;
  constexpr int kind = C < nS ? 0 : C < 2 * nS ? 1 : 2;  // U, V, P
  constexpr int cl = kind == 0 ? C : kind == 1 ? C - nS : C - 2 * nS;
  constexpr int kk = cl * 32 + k;
  if constexpr (kind < 2) {
    if constexpr (kk >= 2 * P) {
      return 0.0f;
    } else {
      constexpr int d = kk / P, pr = kk % P;
      constexpr int j = pair_j(pr), i = pr - j * (j + 1) / 2;
      const float(&S)[K] = kind == 0 ? U : V;
      const float(&w)[K] = d == 0 ? uc : vc;
      if constexpr (i == j) return S[i] * w[i];
      else return fmaf(S[i], w[j], S[j] * w[i]);
    }
  } else {
    if constexpr (kk >= P) {
      return 0.0f;
    } else {
      constexpr int j = pair_j(kk), i = kk - j * (j + 1) / 2;
      if constexpr (i == j) return xi[i] * pp[i];
      else return fmaf(xi[i], pp[j], xi[j] * pp[i]);
    }
  }
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
  constexpr int RS = tc_RS(K), RP = tc_RP(K);
  constexpr int nS = RS / 32, nP = RP / 32, NC = 2 * nS + nP;
  constexpr int BFL = tc_bfloats(K);
  constexpr int ABUF = TC_M * 32;  // floats of one part of one A chunk
  constexpr int NB = tc_nbuf(K);
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  float* sB = reinterpret_cast<float*>(tc_smem_raw);
  float* sA = sB + BFL;  // [NB buffers][head, tail][ABUF]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + NB * TC_PARTS * ABUF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  const int t = threadIdx.x, w = t >> 5;
  const uint32_t bar_b = smem_u32(&bars[0]);
  const uint32_t bar_f[2] = {smem_u32(&bars[1]), smem_u32(&bars[2])};

  if (t == 0) {
    mbar_init(bar_b, 1);
    mbar_init(bar_f[0], 1);
    mbar_init(bar_f[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (t == 0) {  // B image: one bulk TMA copy global -> shared
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(bar_b), "r"((uint32_t)(BFL * 4))
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(sB)),
        "l"(bimg), "r"((uint32_t)(BFL * 4)), "r"(bar_b)
        : "memory");
  }

  // this thread's element
  const int64_t l = (int64_t)blockIdx.x * TC_M + t;
  const bool live = l < n;
  const int64_t e = g0 + (live ? l : 0), ne = m.ne;
  const float* geo = m.geo32;
  float xi[K], U[K], V[K], uc[K], vc[K], pp[K];
  float J0 = 0.f, J1 = 0.f, J2 = 0.f, J3 = 0.f, rs = 0.f, hb0 = 0.f;
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
    sfor<0, K>([&](auto j) { xi[j] = U[j] = V[j] = uc[j] = vc[j] = pp[j] = 0.0f; });
  }

  bool ok = true;
  sfor<0, NC>([&](auto Cc) {
    constexpr int C = Cc;
    constexpr int b = C % NB;
    float* aH = sA + (TC_PARTS * b) * ABUF;
    float* aT = aH + ABUF;
    if constexpr (C >= NB) ok &= mbar_wait(bar_f[b], (C / NB - 1) & 1);  // MMAs of chunk C - NB done
    sfor<0, 8>([&](auto KQ) {
      float v[4];
      sfor<0, 4>([&](auto KR) { v[KR] = tc_value<K, C, KQ * 4 + KR>(xi, U, V, uc, vc, pp); });
      float4 h4, t4;
      split4(v, h4, t4);
      const int off = (t >> 3) * 256 + KQ * 32 + (t & 7) * 4;
      *reinterpret_cast<float4*>(aH + off) = h4;
      *reinterpret_cast<float4*>(aT + off) = t4;
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      if constexpr (C == 0) ok &= mbar_wait(bar_b, 0);
      tc_fence_after();
      constexpr int kind = C < nS ? 0 : C < 2 * nS ? 1 : 2;
      constexpr int cl = kind == 0 ? C : kind == 1 ? C - nS : C - 2 * nS;
      constexpr uint32_t idesc = kind == 2 ? tc_idesc(TC_M, TC_NP) : tc_idesc(TC_M, TC_NS);
      const uint32_t d = tmem + (kind == 0 ? 0u : kind == 1 ? 16u : 32u);
      const float* bH = kind == 2 ? sB + TC_PARTS * TC_NS * RS + cl * (TC_NP * 32) : sB + cl * (TC_NS * 32);
      const int bpart = kind == 2 ? TC_NP * RP : TC_NS * RS;  // floats between the parts of B
      const uint32_t a0 = smem_u32(aH), b0 = smem_u32(bH);
      const uint32_t ap = ABUF * 4, bp = (uint32_t)bpart * 4;  // bytes between parts
#pragma unroll
      for (int s = 0; s < 4; ++s) {  // K = 8 per MMA: two core matrices (256 B) along k
        const uint32_t o = 256u * s;
        tc_mma(d, tc_desc(a0 + o), tc_desc(b0 + o), idesc, (cl == 0 && s == 0) ? 0u : 1u);  // h h
        tc_mma(d, tc_desc(a0 + o), tc_desc(b0 + bp + o), idesc, 1u);                        // h t
        tc_mma(d, tc_desc(a0 + ap + o), tc_desc(b0 + o), idesc, 1u);                        // t h
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_f[b])
                   : "memory");
    }
  });

  // the last commit covers every MMA of the tile
  constexpr int CL = NC - 1;
  bool done = mbar_wait(bar_f[CL % NB], (CL / NB) & 1);
  ok &= done;
  tc_fence_after();
  float dU[16], dV[16], dPx[16], dPy[16];
  const uint32_t lane_base = tmem + ((uint32_t)(32 * w) << 16);
  tmem_ld16(lane_base + 0, dU);
  tmem_ld16(lane_base + 16, dV);
  tmem_ld16(lane_base + 32, dPx);
  tmem_ld16(lane_base + 48, dPy);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  // The mean mode of h_b is the largest term of the pressure products (depths of
  // kilometres against elevations of metres); it enters only through
  // hb0 * sum_i xi_i G_k[q][i][0], which the CUDA cores add here in FP32, so
  // that the tensor cores' accumulation sees no term of that magnitude.
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
  if (!done) mbar_wait(bar_f[CL % NB], (CL / NB) & 1);  // bounded second wait before TMEM is freed
  tc_fence_before();
  __syncthreads();
  if (w == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
  }
}

static_assert(tc_smem(15) <= 227 * 1024, "shared memory of k_vol_tc<15>");
static_assert(TC_NS * 32 % 256 == 0 && TC_NP * 32 % 256 == 0, "whole row groups per chunk");

template <int K>
static int vol_group(cudaStream_t st, const DevMesh& m, const Groups& G, int p, const Phys& ph, StateDev c, VelDev u,
                     float* vol, unsigned* status, const float* bimg) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  const int64_t nrc = G.start[5] - G.start[2], rc_off = g0 - G.start[2];
  k_vol_tc<K><<<(unsigned)((n + TC_M - 1) / TC_M), TC_M, tc_smem(K), st>>>(
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
  int r = vol_group<6>(st, m, G, 2, ph, c, u, vol, status, bimg);
  if (!r) r = vol_group<10>(st, m, G, 3, ph, c, u, vol, status, bimg);
  if (!r) r = vol_group<15>(st, m, G, 4, ph, c, u, vol, status, bimg);
  return r;
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
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(6)));
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(10)));
  SWE_CUDA_OK(cudaFuncSetAttribute(k_vol_tc<15>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem(15)));
  return 0;
}

}  // namespace corrtc
}  // namespace swedg
