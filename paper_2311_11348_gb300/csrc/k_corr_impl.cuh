// Correction part of the order-separated scheme (Sect. 3, Eq. 13 and the
// text after it): every term with a test index or a coefficient index of
// degree >= 2.  Included by k_corr64.cu (FP64 correction) and k_corr32.cu
// (FP32 correction), which define CORR_T and CORR_NS before including it.
//
//   k_usolve_corr<K>   truncated auxiliary system uH = q for one order group
//                      (K x K symmetric, LDL^T), also writes the degree-1
//                      modes, the element's trace record for the edge kernel,
//                      in the first stage of a CFL step its CFL bound, and
//                      (FP64 and mixed modes) the correction of the base
//                      modes rc (volume terms of the degree-1 test modes)
//   k_edge_corr<PM>    edges with max(p_L, p_R) = PM >= 2: traces of the P1
//                      and higher parts at npts_for(PM) Gauss points, the LF
//                      flux of the higher part written as a sum of products
//                      (no cancellation against the base flux), the full flux
//                      projected onto both sides' higher test modes, and the
//                      two-point equivalent of the correction flux for the
//                      base modes (Fbc)
//   k_elem_corr<K>     volume terms as contractions with the reference
//                      tensors D and G of Eq. (13) (compile-time sparsity),
//                      source, the edges' projected fluxes and the SSP-RK
//                      update of the higher modes (test modes q >= 3); in the
//                      tensor-core mode also the test modes 1, 2 (rc)
//
// With CORR_TC defined (k_corr_tc.cu) the volume terms of the momentum rows
// come from a buffer that the tensor-core contraction k_vol_tc<K> wrote;
// k_elem_corr then computes only the elevation row's volume term itself.
#include <cfloat>
#include <cstdio>

#include "kernels.h"
#include "tables.h"

namespace swedg {
namespace CORR_NS {

using T = CORR_T;
constexpr bool kF32 = sizeof(T) == 4;

// The FP32 correction reads FP32 copies of the base state, velocity and
// geometry (written once per element by the base kernels), so it runs no
// conversions on the FP64 pipe.
__device__ __forceinline__ const T* base_c(const StateDev& s) {
  if constexpr (kF32) return (const T*)s.cb32; else return (const T*)s.cb;
}
__device__ __forceinline__ const T* base_u(const VelDev& u) {
  if constexpr (kF32) return (const T*)u.ub32; else return (const T*)u.ub;
}
__device__ __forceinline__ const T* geo_t(const DevMesh& m) {
  if constexpr (kF32) return (const T*)m.geo32; else return (const T*)m.geo;
}
__device__ __forceinline__ const T* egeo_t(const DevMesh& m) {
  if constexpr (kF32) return (const T*)m.egeo32; else return (const T*)m.egeo;
}

__host__ __device__ constexpr int pk(int i, int j) { return i <= j ? j * (j + 1) / 2 + i : i * (i + 1) / 2 + j; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }
// orthogonality zeros: phi_i is orthogonal to every polynomial of degree < deg i
__host__ __device__ constexpr bool tnz(int n, int i, int j) {
  return deg_of(n) <= deg_of(i) + deg_of(j) && deg_of(i) <= deg_of(n) + deg_of(j) && deg_of(j) <= deg_of(n) + deg_of(i);
}
__host__ __device__ constexpr bool gnz(int q, int i, int j) {
  return deg_of(q) == 0 ? false
         : deg_of(q) == 1 ? i == j
                          : (deg_of(i) <= deg_of(j) + deg_of(q) - 1 && deg_of(j) <= deg_of(i) + deg_of(q) - 1);
}
__host__ __device__ constexpr bool dnz(int q, int i) { return deg_of(i) < deg_of(q) && (deg_of(q) != 1 || i == 0); }
__host__ __device__ constexpr bool base2(int q, int i) { return q < 3 && i < 3; }
__host__ __device__ constexpr bool base3(int q, int i, int j) { return q < 3 && i < 3 && j < 3; }
// truncation of the auxiliary system (Sect. 3): K(max(deg i, deg j))
__host__ __device__ constexpr int ktr(int i, int j) { return Kof(imax(deg_of(i), deg_of(j))); }

__constant__ T cT[KMAX][120];       // T[n][i][j], (i, j) packed symmetric
__constant__ T cG[2][KMAX][120];    // G_k[q][i][j], (i, j) packed symmetric
__constant__ T cD[2][KMAX][KMAX];   // D_k[q][i]
__constant__ T cEB[3][3][KMAX][8];  // per PM-2: phihat_i(gamma_k(s_g)) at npts_for(PM) points
__constant__ T cEW[3][8];           // weights on [0,1]
__constant__ T cES[3][8];           // points on [0,1]
__constant__ T cPhi0;
__constant__ T cS2b[2];             // points of the two-point base rule on [0,1]
__constant__ T cRS2b;               // 1 / (s_1 - s_0)
__constant__ double cEV[3][2][3];   // phihat_i(gamma_k(a)), i < 3, at the edge ends a = 0, 1 (FP64 in every mode)

void upload_tables() {
  const RefTables& R = tables();
  static T t[KMAX][120], g[2][KMAX][120], d[2][KMAX][KMAX], eb[3][3][KMAX][8], ew[3][8], es[3][8];
  for (int n = 0; n < KMAX; ++n)
    for (int j = 0; j < KMAX; ++j)
      for (int i = 0; i <= j; ++i) {
        t[n][pk(i, j)] = (T)R.T[n][i][j];
        g[0][n][pk(i, j)] = (T)R.G[0][n][i][j];
        g[1][n][pk(i, j)] = (T)R.G[1][n][i][j];
      }
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < KMAX; ++q)
      for (int i = 0; i < KMAX; ++i) d[k][q][i] = (T)R.D[k][q][i];
  for (int pm = 2; pm <= 4; ++pm) {
    const int N = npts_for(pm);
    for (int gg = 0; gg < 8; ++gg) {
      ew[pm - 2][gg] = gg < N ? (T)R.ew[N][gg] : (T)0;
      es[pm - 2][gg] = gg < N ? (T)R.es[N][gg] : (T)0;
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < KMAX; ++i) eb[pm - 2][k][i][gg] = gg < N ? (T)R.EB[N][k][i][gg] : (T)0;
    }
  }
  const T s2b[2] = {(T)R.es[2][0], (T)R.es[2][1]};
  const T rs2b = (T)(1.0 / (R.es[2][1] - R.es[2][0]));
  cudaMemcpyToSymbol(cS2b, s2b, sizeof s2b);
  cudaMemcpyToSymbol(cRS2b, &rs2b, sizeof rs2b);
  const T phi0 = (T)R.phi0;
  cudaMemcpyToSymbol(cT, t, sizeof t);
  cudaMemcpyToSymbol(cG, g, sizeof g);
  cudaMemcpyToSymbol(cD, d, sizeof d);
  cudaMemcpyToSymbol(cEB, eb, sizeof eb);
  cudaMemcpyToSymbol(cEW, ew, sizeof ew);
  cudaMemcpyToSymbol(cES, es, sizeof es);
  cudaMemcpyToSymbol(cPhi0, &phi0, sizeof phi0);
  cudaMemcpyToSymbol(cEV, R.EV, sizeof R.EV);
}

static inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ double tide_value(const Phys& ph, double t) {
  if (ph.tide_period <= 0.0) return ph.tide_amp;
  return ph.tide_amp * sin(2.0 * 3.14159265358979323846 * t / ph.tide_period + ph.tide_phase);
}

// 16-byte accesses to 4 consecutive values (FP64: two of them)
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}
__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 v = *reinterpret_cast<const double2*>(p), w = *reinterpret_cast<const double2*>(p + 2);
  a = v.x; b = v.y; c = w.x; d = w.y;
}

// Load all K modes of field f (base rows from the FP64 base state, higher rows
// from the group's correction array).
template <int K>
__device__ __forceinline__ void load_modes(T (&out)[K], const T* __restrict__ base, int64_t ne, int64_t e,
                                           const T* __restrict__ high, int64_t n, int64_t l, int f) {
  sfor<0, K>([&](auto i) {
    if constexpr (i < 3) out[i] = base[(f * 3 + i) * ne + e];
    else out[i] = high[(f * (K - 3) + (i - 3)) * n + l];
  });
}

// ---------------------------------------------------------------------------
// Volume terms of Eq. (13) for one test mode Q (non-base index triples only),
// with J^{-1} folded into the contravariant coefficients
//   Uc_i = (J^-1 q_i)_xhat, Vc_i = (J^-1 q_i)_yhat, uc_j, vc_j likewise, pp_j = xi_j/2:
//   r_xi = sum_i Uc_i D_x[Q][i] + Vc_i D_y[Q][i]
//   r_U  = (1/s) [ sum_ij U_i (uc_j G_x[Q][i][j] + vc_j G_y[Q][i][j]) + g (J00 P_x + J10 P_y) ]
//   r_V  = (1/s) [ sum_ij V_i (...) + g (J01 P_x + J11 P_y) ]
//   P_k  = sum_ij xi_i pp_j G_k[Q][i][j] + sum_{i >= 3, j < 3} xi_i hb_j G_k[Q][i][j]
// The bottom term g xi h_b keeps only the products with a higher elevation
// mode i >= 3.  For Q < 3 the rest are base triples.  For Q >= 3 the rest,
// g (xi_lin h_b) with xi_lin the degree-1 part of xi, integrates by parts to
// its own boundary integral (the gradient of xi_lin h_b is linear, so phi_Q
// of degree >= 2 is orthogonal to it): the correction edge kernel moves that
// integral into the edge flux, where it meets the flux's own g xi_lin h_b
// term and leaves g h_b times the jump of xi_lin, formed in FP64.  In FP32
// the two O(g |xi| h_b) integrals otherwise cancel to a residual several
// orders of magnitude smaller and carry their rounding error into it.
// ---------------------------------------------------------------------------
// The structural zeros depend on the degrees of q, i, j only, so one body
// serves every test mode of degree DQ (q a run-time value: the tensors are
// read with a block-uniform index, and K = 15 needs 4 code bodies instead of
// 14, which the instruction cache holds); QR stands for the degree class in
// the compile-time predicates.
template <int DQ>
__host__ __device__ constexpr int qrep() { return DQ <= 1 ? DQ : Kof(DQ - 1); }

template <int K, int DQ, int KL>
__device__ __forceinline__ void volume_c(T (&r)[3], int q, const T (&xi)[K], const T (&U)[K], const T (&V)[K],
                                         const T (&uc)[K], const T (&vc)[K], const T (&pp)[K], const T (&hb)[3],
                                         const T (&Uc)[KL], const T (&Vc)[KL], T rs, T J0, T J1, T J2, T J3,
                                         T g) {
  constexpr int QR = qrep<DQ>();
  T am = 0;
  sfor<0, KL>([&](auto i) {
    if constexpr (dnz(QR, i) && !base2(QR, i)) am += Uc[i] * cD[0][q][i] + Vc[i] * cD[1][q][i];
  });
  T aU = 0, aV = 0, Px = 0, Py = 0;
  sfor<0, K>([&](auto i) {
    constexpr bool any = [] {
      for (int j = 0; j < K; ++j)
        if (gnz(QR, decltype(i)::value, j) && !base3(QR, decltype(i)::value, j)) return true;
      return false;
    }();
    if constexpr (any) {
      T w = 0, px = 0, py = 0;
      sfor<0, K>([&](auto j) {
        if constexpr (gnz(QR, i, j) && !base3(QR, i, j)) {
          const T gx = cG[0][q][pk(i, j)], gy = cG[1][q][pk(i, j)];
          w += uc[j] * gx + vc[j] * gy;
          T pj = pp[j];
          if constexpr (i >= 3 && j < 3) pj += hb[j];
          px += pj * gx;
          py += pj * gy;
        }
      });
      aU += U[i] * w; aV += V[i] * w;
      Px += xi[i] * px; Py += xi[i] * py;
    }
  });
  r[0] = am;
  r[1] = rs * (aU + g * (J0 * Px + J2 * Py));
  r[2] = rs * (aV + g * (J1 * Px + J3 * Py));
}

// one test mode Q known at compile time
template <int K, int Q, int KL>
__device__ __forceinline__ void volume_q(T (&r)[3], const T (&xi)[K], const T (&U)[K], const T (&V)[K],
                                         const T (&uc)[K], const T (&vc)[K], const T (&pp)[K], const T (&hb)[3],
                                         const T (&Uc)[KL], const T (&Vc)[KL], T rs, T J0, T J1, T J2, T J3,
                                         T g) {
  volume_c<K, deg_of(Q), KL>(r, Q, xi, U, V, uc, vc, pp, hb, Uc, Vc, rs, J0, J1, J2, J3, g);
}

// the elevation row of volume_c alone
template <int K, int DQ, int KL>
__device__ __forceinline__ T volume_xi(int q, const T (&Uc)[KL], const T (&Vc)[KL]) {
  constexpr int QR = qrep<DQ>();
  T am = 0;
  sfor<0, KL>([&](auto i) {
    if constexpr (dnz(QR, i) && !base2(QR, i)) am += Uc[i] * cD[0][q][i] + Vc[i] * cD[1][q][i];
  });
  return am;
}

#ifdef CORR_TC
#define CORR_VOL_PARAM , const float* __restrict__ vol
#define CORR_VOL_ARG , vol
// orders whose momentum volume terms come from the tensor cores; for K = 6
// the CUDA-core contraction measured as fast as the tensor-core kernel plus
// the buffer round trip, so it stays here
__host__ __device__ constexpr bool tc_vol(int K) { return K >= 10; }
#else
#define CORR_VOL_PARAM
#define CORR_VOL_ARG
__host__ __device__ constexpr bool tc_vol(int K) { return false; }
#endif

// ---------------------------------------------------------------------------
// auxiliary system of one order group:  M u = U, M v = V,
//   M[i][j] = (1/s) sum_{n < K(max deg)} H_n T[n][i][j],  H = xi + h_b.
// Solved as S u = s U with S = s M by an unpivoted LDL^T factorisation.
// With rc given, the same thread then forms the correction of the base modes
// (the volume terms of the degree-1 test modes with a coefficient of degree
// >= 2) from the velocity it has just solved for, so that the base element
// kernel can take it without waiting for the correction element kernel.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void usolve_corr_body(const DevMesh& m, int64_t g0, int64_t n, const Phys& ph,
                                                 const StateDev& c, const T* __restrict__ ch, double* __restrict__ ub,
                                                 float* __restrict__ ub32, T* __restrict__ uh,
                                                 T* __restrict__ tr, T* __restrict__ trv,
                                                 unsigned* status, unsigned long long* dmin,
                                                 double* __restrict__ rc, int64_t rc_off, int64_t nrc) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dcfl = DBL_MAX;
  int mem = 0;
  if (l < n) {
    const int64_t e = g0 + l, ne = m.ne;
    constexpr int KH = K - 3, NP = K * (K + 1) / 2;
    const T* cb = base_c(c);
    const T* geo = geo_t(m);
    T H[K];
    load_modes<K>(H, cb, ne, e, ch, n, l, 0);
    H[0] += geo[G_HB0 * ne + e];
    H[1] += geo[G_HB1 * ne + e];
    H[2] += geo[G_HB2 * ne + e];
    // depth check on the FP64 mean (base modes are FP64 in every mode)
    const double H0d = c.cb[e] + m.geo[G_HB0 * ne + e];
    if (!(H0d * m.geo[G_RS * ne + e] * 1.4142135623730951 > ph.h_min)) {
      atomicOr(status, (unsigned)ST_DEPTH);
      atomicOr(m.mstatus + m.mem[e], (unsigned)ST_DEPTH);
    }
    const T sv = geo[G_S * ne + e];
    T A[NP];
    sfor<0, K>([&](auto j) {
      sfor<0, j + 1>([&](auto i) {
        T acc = 0;
        sfor<0, ktr(i, j)>([&](auto nn) {
          if constexpr (tnz(nn, i, j)) acc += H[nn] * cT[nn][pk(i, j)];
        });
        A[pk(i, j)] = acc;
      });
    });
    // LDL^T: A[pk(i,j)] (i > j) <- L_ij;  dg[j] = d_j, rd[j] = 1/d_j
    T dg[K], rd[K];
    sfor<0, K>([&](auto j) {
      T dj = A[pk(j, j)];
      sfor<0, j>([&](auto k) { dj -= A[pk(j, k)] * A[pk(j, k)] * dg[k]; });
      dg[j] = dj;
      rd[j] = (T)1 / dj;
      sfor<j + 1, K>([&](auto i) {
        T w = A[pk(i, j)];
        sfor<0, j>([&](auto k) { w -= A[pk(i, k)] * A[pk(j, k)] * dg[k]; });
        A[pk(i, j)] = w * rd[j];
      });
    });
    T x[2][K];
    load_modes<K>(x[0], cb, ne, e, ch, n, l, 1);
    load_modes<K>(x[1], cb, ne, e, ch, n, l, 2);
    const T s = sv;
    double u00 = 0.0, v00 = 0.0;  // mode 0 of u and v as stored (FP64)
    sfor<0, 2>([&](auto r) {
      sfor<0, K>([&](auto i) { sfor<0, i>([&](auto k) { x[r][i] -= A[pk(i, k)] * x[r][k]; }); });
      sfor<0, K>([&](auto i) { x[r][i] *= rd[i]; });
      sfor<0, K>([&](auto ii) {
        constexpr int i = K - 1 - ii;
        sfor<i + 1, K>([&](auto k) { x[r][i] -= A[pk(k, i)] * x[r][k]; });
      });
      sfor<0, K>([&](auto i) {
        const T v = x[r][i] * s;
        if constexpr (i < 3) {
          ub[(r * 3 + i) * ne + e] = (double)v;
          if constexpr (kF32) ub32[(r * 3 + i) * ne + e] = v;
          if constexpr (i == 0) {
            if constexpr (r == 0) u00 = (double)v; else v00 = (double)v;
          }
        } else {
          uh[(r * KH + (i - 3)) * n + l] = v;
        }
      });
    });
    if (dmin) {
      mem = m.mem[e];
      dcfl = cfl_bound(u00, v00, H0d, m.geo[G_RS * ne + e], ph.g, m.geo[G_DIAM * ne + e], m.p[e]);
    }
    T xi[K], U[K], V[K];
    load_modes<K>(xi, cb, ne, e, ch, n, l, 0);
    load_modes<K>(U, cb, ne, e, ch, n, l, 1);
    load_modes<K>(V, cb, ne, e, ch, n, l, 2);
    // this element's trace record for the correction edges (VelDev::tr)
    sfor<0, K>([&](auto i) {
      st4(tr + (l * K + i) * 4, xi[i], U[i], V[i], x[0][i] * s);
      trv[l * K + i] = x[1][i] * s;
    });
    if (rc) {
      constexpr int KL = Kof(deg_of(K - 1) - 1);  // modes of degree < p (the only ones D couples)
      T uc[K], vc[K], pp[K], Uc[KL], Vc[KL];
      const T J0 = geo[G_JI0 * ne + e], J1 = geo[G_JI1 * ne + e];
      const T J2 = geo[G_JI2 * ne + e], J3 = geo[G_JI3 * ne + e];
      const T hb[3] = {geo[G_HB0 * ne + e], geo[G_HB1 * ne + e], geo[G_HB2 * ne + e]};
      sfor<0, K>([&](auto j) {
        const T uu = x[0][j] * s, vv = x[1][j] * s;  // the velocity modes as stored above
        uc[j] = J0 * uu + J1 * vv;
        vc[j] = J2 * uu + J3 * vv;
        pp[j] = (T)0.5 * xi[j];
        if constexpr (j < KL) {
          Uc[j] = J0 * U[j] + J1 * V[j];
          Vc[j] = J2 * U[j] + J3 * V[j];
        }
      });
      const T rs = geo[G_RS * ne + e], g = (T)ph.g;
      T r1[3], r2[3];
      volume_q<K, 1, KL>(r1, xi, U, V, uc, vc, pp, hb, Uc, Vc, rs, J0, J1, J2, J3, g);
      volume_q<K, 2, KL>(r2, xi, U, V, uc, vc, pp, hb, Uc, Vc, rs, J0, J1, J2, J3, g);
      rc[0 * nrc + rc_off + l] = (double)r1[1];
      rc[1 * nrc + rc_off + l] = (double)r2[1];
      rc[2 * nrc + rc_off + l] = (double)r1[2];
      rc[3 * nrc + rc_off + l] = (double)r2[2];
    }
  }
  if (dmin) cfl_min_store(dmin, mem, dcfl);  // uniform over the grid: every lane of the warp is here
}

// The compiler's register allocation (FP32: 80, 127, 255 registers for K =
// 6, 10, 15), and for K = 15 in FP32 a second build in 168 registers (3
// blocks per SM) for launch shapes that cap the base grids (see k_edge_corr).
template <int K>
__global__ void __launch_bounds__(128) k_usolve_corr(DevMesh m, int64_t g0, int64_t n, Phys ph, StateDev c,
                                                     const T* __restrict__ ch, double* __restrict__ ub,
                                                     float* __restrict__ ub32, T* __restrict__ uh,
                                                     T* __restrict__ tr, T* __restrict__ trv,
                                                     unsigned* status, unsigned long long* dmin,
                                                     double* __restrict__ rc, int64_t rc_off, int64_t nrc) {
  usolve_corr_body<K>(m, g0, n, ph, c, ch, ub, ub32, uh, tr, trv, status, dmin, rc, rc_off, nrc);
}
__global__ void __launch_bounds__(128, 3) k_usolve_corr15(DevMesh m, int64_t g0, int64_t n, Phys ph, StateDev c,
                                                         const T* __restrict__ ch, double* __restrict__ ub,
                                                         float* __restrict__ ub32, T* __restrict__ uh,
                                                         T* __restrict__ tr, T* __restrict__ trv,
                                                         unsigned* status, unsigned long long* dmin,
                                                         double* __restrict__ rc, int64_t rc_off, int64_t nrc) {
  usolve_corr_body<15>(m, g0, n, ph, c, ch, ub, ub32, uh, tr, trv, status, dmin, rc, rc_off, nrc);
}

template <int K>
static int usolve_group(cudaStream_t st, const DevMesh& m, const Groups& G, int p, const Phys& ph, StateDev c,
                        VelDev u, unsigned* status, unsigned long long* dmin, void* rc) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  const int64_t nrc = G.start[5] - G.start[2], rc_off = g0 - G.start[2];
  const int ct = launch_shape().corr_threads;
  if (K == 15 && kF32 && launch_shape().base_bpsm > 0)
    k_usolve_corr15<<<nblocks(n, ct), ct, 0, st>>>(m, g0, n, ph, c, (const T*)c.ch[p], u.ub, u.ub32,
                                                   (T*)u.uh[p], (T*)u.tr[p], (T*)u.trv[p], status, dmin,
                                                   (double*)rc, rc_off, nrc);
  else
    k_usolve_corr<K><<<nblocks(n, ct), ct, 0, st>>>(m, g0, n, ph, c, (const T*)c.ch[p], u.ub, u.ub32,
                                                      (T*)u.uh[p], (T*)u.tr[p], (T*)u.trv[p], status, dmin,
                                                      (double*)rc, rc_off, nrc);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_usolve_corr(GroupStreams gs, const DevMesh& m, const Groups& G, const Phys& ph, StateDev c, VelDev u,
                       unsigned* status, unsigned long long* dmin, void* rc) {
  int r = usolve_group<6>(gs.s[0], m, G, 2, ph, c, u, status, dmin, rc);
  if (!r) r = usolve_group<10>(gs.s[1], m, G, 3, ph, c, u, status, dmin, rc);
  if (!r) r = usolve_group<15>(gs.s[2], m, G, 4, ph, c, u, status, dmin, rc);
  return r;
}

// ---------------------------------------------------------------------------
// correction edge flux.  Per side the traces are split into the P1 part (b)
// and the higher part (h).  With w = u.n, P = g xi (xi/2 + h_b):
//   A.n(b+h) - A.n(b) = ( U_h nx + V_h ny,
//                         U_h w + U_b w_h + g nx xi_h (xi_b + xi_h/2 + h_b),
//                         V_h w + V_b w_h + g ny xi_h (xi_b + xi_h/2 + h_b) )
// so the correction flux  F_h = 1/2 (A_h(L) + A_h(R) + lambda (c_h(L) - c_h(R)))
// carries no cancellation against the base flux.  F_f = F_b + F_h is the LF
// flux the test modes of degree >= 2 see, except that the g xi_lin h_b terms
// of F_b give way to g h_b times the jump of xi_lin (the volume term's share,
// see volume_q).  Both are stored pre-weighted by |E| w_g at the points of
// the left element's direction.
// ---------------------------------------------------------------------------
struct Tr { T xb, Ub, Vb, ub, vb, xh, Uh, Vh, uh, vh; };

template <int PM>
__device__ __forceinline__ void side_traces(const DevMesh& m, const Groups& G, StateDev c, VelDev u, int64_t e,
                                            int p, int k, bool reverse, Tr (&tr)[npts_for(PM)]) {
  constexpr int N = npts_for(PM), KM = Kof(PM), GI = PM - 2;
  const int64_t ne = m.ne;
  const int K = Kof(p);
  const T rs = geo_t(m)[G_RS * ne + e];
  const T* cbt = base_c(c);
  const T* ubt = base_u(u);
  // an element of order >= 2 reads its trace record (16 + 4 bytes per mode),
  // an element of order <= 1 its base modes from the base state and velocity
  const T* r4 = nullptr;
  const T* rv = nullptr;
  if (p >= 2) {  // selects, not a runtime index into the parameter arrays (that would copy them to the stack)
    const int64_t s0 = p == 2 ? G.start[2] : p == 3 ? G.start[3] : G.start[4];
    const int64_t l = e - s0;
    r4 = (const T*)(p == 2 ? u.tr[2] : p == 3 ? u.tr[3] : u.tr[4]) + l * K * 4;
    rv = (const T*)(p == 2 ? u.trv[2] : p == 3 ? u.trv[3] : u.trv[4]) + l * K;
  }
  sfor<0, N>([&](auto g) { tr[g] = Tr{0, 0, 0, 0, 0, 0, 0, 0, 0, 0}; });
  sfor<0, KM>([&](auto i) {
    if (i >= K) return;
    T cx, cU, cV, cu, cv;
    if (p >= 2) {
      ld4(r4 + i * 4, cx, cU, cV, cu);
      cv = rv[i];
    } else if constexpr (i < 3) {
      cx = cbt[(0 * 3 + i) * ne + e]; cU = cbt[(1 * 3 + i) * ne + e]; cV = cbt[(2 * 3 + i) * ne + e];
      cu = ubt[(0 * 3 + i) * ne + e]; cv = ubt[(1 * 3 + i) * ne + e];
    }
    sfor<0, N>([&](auto g) {
      const T b = rs * (reverse ? cEB[GI][k][i][N - 1 - g] : cEB[GI][k][i][g]);
      if constexpr (i < 3) {
        tr[g].xb += cx * b; tr[g].Ub += cU * b; tr[g].Vb += cV * b; tr[g].ub += cu * b; tr[g].vb += cv * b;
      } else {
        tr[g].xh += cx * b; tr[g].Uh += cU * b; tr[g].Vh += cV * b; tr[g].uh += cu * b; tr[g].vh += cv * b;
      }
    });
  });
}

template <int PM>
__device__ __forceinline__ void edge_corr_body(const DevMesh& m, const int32_t* __restrict__ list, int64_t nl,
                                               const Groups& G, const Phys& ph, const Stage& stg, const StateDev& c,
                                               const VelDev& u, double* __restrict__ Fbc, const EdgeFlux& fx) {
  constexpr int N = npts_for(PM), GI = PM - 2;
  void* const* Pf = fx.Pf;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nl) return;
  const int64_t ed = list[idx], nE = m.nedge;
  const int L = m.eL[ed], R = m.eR[ed], info = m.einfo[ed];
  const int kL = info & 3, kR = (info >> 2) & 3, bc = info >> 4;
  const int pL = m.p[L], pR = R >= 0 ? m.p[R] : 0;
  const T* eg = egeo_t(m);
  const T len = eg[E_LEN * nE + ed], nx = eg[E_NX * nE + ed], ny = eg[E_NY * nE + ed];
  const T hA = eg[E_HA * nE + ed], hB = eg[E_HB * nE + ed];
  const T g = (T)ph.g;
  const T hmid = eg[E_HMID * nE + ed];
  // lambda of Eq. (10) from the element means (Sect. 3), as in the base flux
  const T* cbt = base_c(c);
  const T* ubt = base_u(u);
  const T* geo = geo_t(m);
  const int64_t ne = m.ne;
  const T mL = (T)1.4142135623730951 * geo[G_RS * ne + L];
  const T unL = (ubt[L] * nx + ubt[3 * ne + L] * ny) * mL;
  const T HL = cbt[L] * mL + hmid;
  T unR, HR;
  double xt = 0.0;  // open sea elevation
  Tr a[N], b[N];
  side_traces<PM>(m, G, c, u, L, pL, kL, false, a);
  if (R >= 0) {
    side_traces<PM>(m, G, c, u, R, pR, kR, true, b);
    const T mR = (T)1.4142135623730951 * geo[G_RS * ne + R];
    unR = (ubt[R] * nx + ubt[3 * ne + R] * ny) * mR;
    HR = cbt[R] * mR + hmid;
  } else if (bc == 2) {
    xt = tide_value(ph, stage_time(stg, m.emem[ed]));
    const T xh = (T)xt;
    sfor<0, N>([&](auto q) { b[q] = a[q]; b[q].xb = xh; b[q].xh = 0; });
    unR = unL;
    HR = xh + hmid;
  } else {
    unR = -unL;
    HR = HL;
    sfor<0, N>([&](auto q) {
      const Tr& t = a[q];
      const T qb = t.Ub * nx + t.Vb * ny, qh = t.Uh * nx + t.Vh * ny;
      const T wb = t.ub * nx + t.vb * ny, wh = t.uh * nx + t.vh * ny;
      b[q] = Tr{t.xb, t.Ub - 2 * qb * nx, t.Vb - 2 * qb * ny, t.ub - 2 * wb * nx, t.vb - 2 * wb * ny,
                t.xh, t.Uh - 2 * qh * nx, t.Vh - 2 * qh * ny, t.uh - 2 * wh * nx, t.vh - 2 * wh * ny};
    });
  }
  const T lam = fmax(fabs(unL), fabs(unR)) + sqrt(g * fmax(HL, HR));
  // jump xi_lin,R - xi_lin,L of the degree-1 elevations at the edge ends
  // (s = 0, 1 of the left element's parameter; the right element runs the
  // edge the other way) from the FP64 base modes: it carries the volume
  // term g xi_lin h_b of the higher test modes (moved here, see volume_q),
  // zero on land, where the mirror state has the same elevation
  double JA = 0.0, JB = 0.0;
  if (R >= 0 || bc == 2) {
    const double rl = m.geo[G_RS * ne + L];
    double lA = 0.0, lB = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lA += c.cb[i * ne + L] * cEV[kL][0][i];
      lB += c.cb[i * ne + L] * cEV[kL][1][i];
    }
    double rA = xt, rB = xt;
    if (R >= 0) {
      const double rr = m.geo[G_RS * ne + R];
      rA = rB = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        rA += c.cb[i * ne + R] * cEV[kR][1][i];
        rB += c.cb[i * ne + R] * cEV[kR][0][i];
      }
      rA *= rr;
      rB *= rr;
    }
    JA = rA - rl * lA;
    JB = rB - rl * lB;
  }
  const T JA_ = (T)JA, dJ = (T)(JB - JA);
  // zeroth and first moments (in the left element's edge parameter s) of the
  // weighted correction flux: they are all the test modes of degree <= 1 see
  T M0[3] = {0, 0, 0}, M1[3] = {0, 0, 0};
  T Ffull[3][N], FJ[N];
  sfor<0, N>([&](auto q) {
    const T hb = hA + cES[GI][q] * (hB - hA);
    const Tr& x = a[q];
    const Tr& y = b[q];
    // base flux (P1 parts, which the base modes take from the base edge
    // kernel): for the higher modes g h_b J replaces its g xi_lin h_b terms
    const T wxb = x.ub * nx + x.vb * ny, wyb = y.ub * nx + y.vb * ny;
    const T pxb = g * x.xb * ((T)0.5 * x.xb), pyb = g * y.xb * ((T)0.5 * y.xb);
    const T Fb0 = (x.Ub + y.Ub) * nx + (x.Vb + y.Vb) * ny + lam * (x.xb - y.xb);
    const T Fb1 = x.Ub * wxb + y.Ub * wyb + (pxb + pyb) * nx + lam * (x.Ub - y.Ub);
    const T Fb2 = x.Vb * wxb + y.Vb * wyb + (pxb + pyb) * ny + lam * (x.Vb - y.Vb);
    // higher part as a sum of products
    const T wxh = x.uh * nx + x.vh * ny, wyh = y.uh * nx + y.vh * ny;
    const T pxh = g * x.xh * (x.xb + (T)0.5 * x.xh + hb), pyh = g * y.xh * (y.xb + (T)0.5 * y.xh + hb);
    const T Fh0 = (x.Uh + y.Uh) * nx + (x.Vh + y.Vh) * ny + lam * (x.xh - y.xh);
    const T Fh1 = x.Uh * (wxb + wxh) + x.Ub * wxh + y.Uh * (wyb + wyh) + y.Ub * wyh + (pxh + pyh) * nx +
                  lam * (x.Uh - y.Uh);
    const T Fh2 = x.Vh * (wxb + wxh) + x.Vb * wxh + y.Vh * (wyb + wyh) + y.Vb * wyh + (pxh + pyh) * ny +
                  lam * (x.Vh - y.Vh);
    const T wgt = (T)0.5 * len * cEW[GI][q];
    const T h0 = wgt * Fh0, h1 = wgt * Fh1, h2 = wgt * Fh2;
    M0[0] += h0; M0[1] += h1; M0[2] += h2;
    M1[0] += h0 * cES[GI][q]; M1[1] += h1 * cES[GI][q]; M1[2] += h2 * cES[GI][q];
    Ffull[0][q] = wgt * (Fb0 + Fh0);
    Ffull[1][q] = wgt * (Fb1 + Fh1);
    Ffull[2][q] = wgt * (Fb2 + Fh2);
    FJ[q] = wgt * g * hb * (JA_ + cES[GI][q] * dJ);
  });
  // the full flux projected onto the higher test modes of each side once here,
  //   P[k][f][q] = -+ (1/s) sum_g (F_f(s_g) +- n_f FJ(s_g)) phihat_q(gamma_k(s_g)),
  // (left: minus, points in its own direction, +J; right: plus, points
  // reversed, -J), stored in the element's own slot of its order group (local
  // edge k), so that the element kernel reads one value per edge, field and
  // mode, consecutive elements contiguous
  auto project = [&](int side, int64_t el, int k, int pside, T sg) {
    const int Kside = Kof(pside), KH = Kside - 3;
    const int64_t s0 = pside == 2 ? G.start[2] : pside == 3 ? G.start[3] : G.start[4];
    const int64_t ns = (pside == 2 ? G.start[3] : pside == 3 ? G.start[4] : G.start[5]) - s0;
    T* P = (T*)(pside == 2 ? Pf[2] : pside == 3 ? Pf[3] : Pf[4]) + (el - s0);
    const T jx = side ? -nx : nx, jy = side ? -ny : ny;
    sfor<3, Kof(PM)>([&](auto q) {
      if (q < Kside) {
        T acc[3] = {0, 0, 0}, aj = 0;
        sfor<0, N>([&](auto g) {
          const T bq = side ? cEB[GI][k][q][N - 1 - g] : cEB[GI][k][q][g];
          acc[0] += Ffull[0][g] * bq;
          acc[1] += Ffull[1][g] * bq;
          acc[2] += Ffull[2][g] * bq;
          aj += FJ[g] * bq;
        });
        P[((k * 3 + 0) * KH + (q - 3)) * ns] = sg * acc[0];
        P[((k * 3 + 1) * KH + (q - 3)) * ns] = sg * (acc[1] + jx * aj);
        P[((k * 3 + 2) * KH + (q - 3)) * ns] = sg * (acc[2] + jy * aj);
      }
    });
  };
  if (pL >= 2) project(0, L, kL, pL, -geo[G_RS * ne + L]);
  if (R >= 0 && pR >= 2) project(1, R, kR, pR, geo[G_RS * ne + R]);
  // Degree-<=1 test functions are linear along the edge, so the correction's
  // share of the base modes is fixed by (M0, M1); the two-point flux with the
  // same moments is stored next to the base flux of this edge, and both sides
  // project their sum in FP64 (one value per edge: conservative in every mode).
  sfor<0, 3>([&](auto f) {
    const T f1 = (M1[f] - cS2b[0] * M0[f]) * cRS2b;
    const T f0 = M0[f] - f1;
    Fbc[(f * 2 + 0) * nE + ed] = (double)f0;
    Fbc[(f * 2 + 1) * nE + ed] = (double)f1;
  });
}

// Register budgets: the compiler's allocation (FP32: 124, 168, 210 registers
// for pmax = 2, 3, 4), and in FP32 second builds for pmax = 3 in 128 and for
// pmax = 4 in 168 registers (4 and 3 blocks per SM) for launch shapes that
// cap the base grids: where the correction kernels share the SMs with a few
// base blocks, the extra warps pay (with the K = 15 velocity solve in 168
// registers, measured on the p 1-4 shelf: -2.6 % per step); beside uncapped
// base grids they do not.
template <int PM>
__global__ void __launch_bounds__(128) k_edge_corr(DevMesh m, const int32_t* __restrict__ list, int64_t nl, Groups G,
                                                   Phys ph, Stage stg, StateDev c, VelDev u,
                                                   double* __restrict__ Fbc, EdgeFlux fx) {
  edge_corr_body<PM>(m, list, nl, G, ph, stg, c, u, Fbc, fx);
}
__global__ void __launch_bounds__(128, 3) k_edge_corr4(DevMesh m, const int32_t* __restrict__ list, int64_t nl,
                                                       Groups G, Phys ph, Stage stg, StateDev c, VelDev u,
                                                       double* __restrict__ Fbc, EdgeFlux fx) {
  edge_corr_body<4>(m, list, nl, G, ph, stg, c, u, Fbc, fx);
}
__global__ void __launch_bounds__(128, 4) k_edge_corr3(DevMesh m, const int32_t* __restrict__ list, int64_t nl,
                                                       Groups G, Phys ph, Stage stg, StateDev c, VelDev u,
                                                       double* __restrict__ Fbc, EdgeFlux fx) {
  edge_corr_body<3>(m, list, nl, G, ph, stg, c, u, Fbc, fx);
}

template <int PM>
static int edge_group(cudaStream_t st, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                      const Stage& stg, StateDev c, VelDev u, EdgeFlux fx) {
  const int64_t nl = ce.n[PM];
  if (nl == 0) return 0;
  const int ct = launch_shape().corr_threads;
  if (PM == 3 && kF32 && launch_shape().base_bpsm > 0)
    k_edge_corr3<<<nblocks(nl, ct), ct, 0, st>>>(m, ce.list[PM], nl, G, ph, stg, c, u, fx.Fbc, fx);
  else if (PM == 4 && kF32 && launch_shape().base_bpsm > 0)
    k_edge_corr4<<<nblocks(nl, ct), ct, 0, st>>>(m, ce.list[PM], nl, G, ph, stg, c, u, fx.Fbc, fx);
  else
    k_edge_corr<PM><<<nblocks(nl, ct), ct, 0, st>>>(m, ce.list[PM], nl, G, ph, stg, c, u, fx.Fbc, fx);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_edge_corr(GroupStreams gs, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                     const Stage& stg, StateDev c, VelDev u, EdgeFlux fx) {
  int r = edge_group<2>(gs.s[0], m, ce, G, ph, stg, c, u, fx);
  if (!r) r = edge_group<3>(gs.s[1], m, ce, G, ph, stg, c, u, fx);
  if (!r) r = edge_group<4>(gs.s[2], m, ce, G, ph, stg, c, u, fx);
  return r;
}


// ---------------------------------------------------------------------------
// correction element update of one order group (K = K(p), p >= 2).
// Block = 128 elements of one test mode q: the grid is ordered q-major
// (blocks 0..nb-1 compute q = 1, the next nb q = 2, ...), so the blocks that
// run at the same time on an SM mostly share one branch of the specialised
// code, and there is one branch per degree of q (volume_c), not per test
// mode: the branches of all test modes do not fit the instruction cache
// (ncu: no_instruction stalls).  q = 1, 2: the correction of the base
// modes (volume terms with a higher coefficient index) -> rc;  q >= 3: the
// full volume term, the source g grad h_b xi_q, the projections of the full
// edge fluxes, and the SSP-RK combination of that higher mode.  One launch
// covers the test modes qlo .. qlo + gridDim.x / nb - 1.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(128, kF32 ? 4 : 2) k_elem_corr(DevMesh m, CorrEdges ce, int64_t g0, int64_t n,
                                                            int64_t rc_off, int64_t nrc, int qlo, Phys ph, Stage stg,
                                                            const T* __restrict__ cbS,
                                                            const T* __restrict__ chS, const T* __restrict__ chN,
                                                            T* __restrict__ chO, const T* __restrict__ ub,
                                                            const T* __restrict__ uh, const T* __restrict__ pe,
                                                            double* __restrict__ rc CORR_VOL_PARAM) {
  const int64_t nb = (n + 127) / 128;
  const int q = qlo + (int)(blockIdx.x / nb);
  const int64_t l = (blockIdx.x % nb) * 128 + threadIdx.x;
  if (l >= n) return;
  const int64_t e = g0 + l, ne = m.ne;
  constexpr int KH = K - 3;
  constexpr int KL = Kof(deg_of(K - 1) - 1);  // modes of degree < p (the only ones D couples)
  const T* geo = geo_t(m);
  const T J0 = geo[G_JI0 * ne + e], J1 = geo[G_JI1 * ne + e];
  const T J2 = geo[G_JI2 * ne + e], J3 = geo[G_JI3 * ne + e];
  const T rs = geo[G_RS * ne + e];
  const T g = (T)ph.g;
  T r[3] = {0, 0, 0};
  // the test mode's own coefficients and the element's mean elevation
  T xq = 0, Uq = 0, Vq = 0, xi0 = 0;
  if constexpr (tc_vol(K)) {
#ifdef CORR_TC
    // the momentum volume terms come from the tensor cores: only the xi row's
    // contravariant momenta (modes of degree < p) are needed here
    T Uc[KL], Vc[KL];
    sfor<0, KL>([&](auto j) {
      T Uj, Vj;
      if constexpr (j < 3) {
        Uj = cbS[(1 * 3 + j) * ne + e];
        Vj = cbS[(2 * 3 + j) * ne + e];
      } else {
        Uj = chS[(1 * KH + (j - 3)) * n + l];
        Vj = chS[(2 * KH + (j - 3)) * n + l];
      }
      Uc[j] = J0 * Uj + J1 * Vj;
      Vc[j] = J2 * Uj + J3 * Vj;
    });
    sfor<1, deg_of(K - 1) + 1>([&](auto DQ) {
      if (deg_of(q) == DQ) r[0] = volume_xi<K, DQ, KL>(q, Uc, Vc);
    });
    r[1] = (T)vol[q * nrc + rc_off + l];
    r[2] = (T)vol[(16 + q) * nrc + rc_off + l];
    if (q >= 3) {
      xq = chS[(0 * KH + (q - 3)) * n + l];
      Uq = chS[(1 * KH + (q - 3)) * n + l];
      Vq = chS[(2 * KH + (q - 3)) * n + l];
    }
    xi0 = cbS[e];
#endif
  } else {
    T xi[K], U[K], V[K], uc[K], vc[K], pp[K], Uc[KL], Vc[KL];
    T uu[K], vv[K];
    load_modes<K>(xi, cbS, ne, e, chS, n, l, 0);
    load_modes<K>(U, cbS, ne, e, chS, n, l, 1);
    load_modes<K>(V, cbS, ne, e, chS, n, l, 2);
    load_modes<K>(uu, ub, ne, e, uh, n, l, 0);
    load_modes<K>(vv, ub, ne, e, uh, n, l, 1);
    const T hb[3] = {geo[G_HB0 * ne + e], geo[G_HB1 * ne + e], geo[G_HB2 * ne + e]};
    sfor<0, K>([&](auto j) {
      uc[j] = J0 * uu[j] + J1 * vv[j];
      vc[j] = J2 * uu[j] + J3 * vv[j];
      pp[j] = (T)0.5 * xi[j];
      if constexpr (j < KL) {
        Uc[j] = J0 * U[j] + J1 * V[j];
        Vc[j] = J2 * U[j] + J3 * V[j];
      }
    });
    sfor<1, deg_of(K - 1) + 1>([&](auto DQ) {
      if (deg_of(q) == DQ) volume_c<K, DQ, KL>(r, q, xi, U, V, uc, vc, pp, hb, Uc, Vc, rs, J0, J1, J2, J3, g);
    });
    sfor<3, K>([&](auto Q) {
      if (q == Q) { xq = xi[Q]; Uq = U[Q]; Vq = V[Q]; }
    });
    xi0 = xi[0];
  }
  if (q < 3) {
    rc[(0 * 2 + (q - 1)) * nrc + rc_off + l] = (double)r[1];
    rc[(1 * 2 + (q - 1)) * nrc + rc_off + l] = (double)r[2];
    return;
  }
  r[1] += geo[G_GDHX * ne + e] * xq;
  r[2] += geo[G_GDHY * ne + e] * xq;
  if (ph.src) {  // bottom friction (tau from the element means, Sect. 3) and Coriolis of Eq. (5)
    const T ra = (T)1.4142135623730951 * rs;
    const T Hm = (xi0 + geo[G_HB0 * ne + e]) * ra;
    const T um = ub[0 * ne + e] * ra, vm = ub[3 * ne + e] * ra;  // mode 0 of u, v (layout [2][3][ne])
    const T tau = (T)ph.fric_lin * Hm + (T)ph.fric_quad * sqrt(um * um + vm * vm);
    const T uq = uh[(0 * KH + (q - 3)) * n + l], vq = uh[(1 * KH + (q - 3)) * n + l];
    r[1] += (T)ph.f_c * Vq - tau * uq;
    r[2] -= (T)ph.f_c * Uq + tau * vq;
  }
  // edges: every edge of a p >= 2 element is a correction edge, whose kernel
  // left the projections in this element's slots
  {
    const T* P = pe + (q - 3) * n + l;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int f = 0; f < 3; ++f) r[f] += P[(k * 3 + f) * KH * n];
  }
  const T dt = (T)stage_dt(stg, m.mem[e]), a = (T)stg.a, b = (T)stg.b;
  const T cs3[3] = {xq, Uq, Vq};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const int64_t ix = (f * KH + (q - 3)) * n + l;
    chO[ix] = stg.rhs_only ? r[f] : (stg.a != 0.0 ? a * chN[ix] : (T)0) + b * (cs3[f] + dt * r[f]);
  }
}

static const T* base_c_host(const StateDev& s) {
  if constexpr (kF32) return (const T*)s.cb32; else return (const T*)s.cb;
}
static const T* base_u_host(const VelDev& u) {
  if constexpr (kF32) return (const T*)u.ub32; else return (const T*)u.ub;
}

template <int K>
static int elem_group(cudaStream_t st, const DevMesh& m, const CorrEdges& ce, const Groups& G, int p, const Phys& ph,
                      const Stage& stg, StateDev cS, StateDev cN, StateDev cO, VelDev u, EdgeFlux fx,
                      void* rc, int part CORR_VOL_PARAM) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  const int64_t nrc = G.start[5] - G.start[2], rc_off = g0 - G.start[2];
  // part 0: every test mode 1 .. K - 1 (rc included); part 1: the higher test modes 3 .. K - 1
  const int qlo = part == 0 ? 1 : 3, nq = part == 0 ? K - 1 : K - 3;
  k_elem_corr<K><<<(unsigned)(((n + 127) / 128) * nq), 128, 0, st>>>(m, ce, g0, n, rc_off, nrc, qlo, ph, stg, base_c_host(cS),
                                                           (const T*)cS.ch[p], (const T*)cN.ch[p], (T*)cO.ch[p],
                                                           base_u_host(u), (const T*)u.uh[p], (const T*)fx.Pf[p],
                                                           (double*)rc CORR_VOL_ARG);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_elem_corr(GroupStreams gs, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                     const Stage& stg, StateDev cS, StateDev cN, StateDev cO, VelDev u, EdgeFlux fx,
                     void* rc, int part CORR_VOL_PARAM) {
  int r = elem_group<6>(gs.s[0], m, ce, G, 2, ph, stg, cS, cN, cO, u, fx, rc, part CORR_VOL_ARG);
  if (!r) r = elem_group<10>(gs.s[1], m, ce, G, 3, ph, stg, cS, cN, cO, u, fx, rc, part CORR_VOL_ARG);
  if (!r) r = elem_group<15>(gs.s[2], m, ce, G, 4, ph, stg, cS, cN, cO, u, fx, rc, part CORR_VOL_ARG);
  return r;
}

}  // namespace CORR_NS
}  // namespace swedg
