// Correction part of the order-separated scheme (Sect. 3, Eq. 13 and the
// text after it): every term with a test index or a coefficient index of
// degree >= 2.  Included by k_corr64.cu (FP64 correction) and k_corr32.cu
// (FP32 correction), which define CORR_T and CORR_NS before including it.
//
//   k_usolve_corr<K>   truncated auxiliary system uH = q for one order group
//                      (K x K symmetric, LDL^T), also writes the degree-1 modes
//   k_edge_corr<PM>    edges with max(p_L, p_R) = PM >= 2: traces of the P1
//                      and higher parts at npts_for(PM) Gauss points, the LF
//                      flux of the higher part written as a sum of products
//                      (no cancellation against the base flux), plus the full
//                      flux for the higher test modes
//   k_elem_corr<K>     volume terms as contractions with the reference
//                      tensors D and G of Eq. (13) (compile-time sparsity),
//                      source, projection of the correction edge fluxes, the
//                      correction of the base modes (rc) and the SSP-RK
//                      update of the higher modes
//   k_elem_corr_lo     p <= 1 elements touching a correction edge: rc only
#include <cstdio>

#include "kernels.h"
#include "tables.h"

namespace swedg {
namespace CORR_NS {

using T = CORR_T;

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
__constant__ double cEBd[3][3][3][8];  // the q < 3 rows of cEB in FP64 (conservative base-mode projection)

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
  static double ebd[3][3][3][8];
  for (int pm = 2; pm <= 4; ++pm)
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i)
        for (int gg = 0; gg < 8; ++gg) ebd[pm - 2][k][i][gg] = gg < npts_for(pm) ? R.EB[npts_for(pm)][k][i][gg] : 0.0;
  cudaMemcpyToSymbol(cEBd, ebd, sizeof ebd);
  const T phi0 = (T)R.phi0;
  cudaMemcpyToSymbol(cT, t, sizeof t);
  cudaMemcpyToSymbol(cG, g, sizeof g);
  cudaMemcpyToSymbol(cD, d, sizeof d);
  cudaMemcpyToSymbol(cEB, eb, sizeof eb);
  cudaMemcpyToSymbol(cEW, ew, sizeof ew);
  cudaMemcpyToSymbol(cES, es, sizeof es);
  cudaMemcpyToSymbol(cPhi0, &phi0, sizeof phi0);
}

static inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ double stage_dt(const Stage& st) { return st.dt ? *st.dt : st.dt_host; }
__device__ __forceinline__ double stage_time(const Stage& st) {
  return (st.t_dev ? *st.t_dev : st.t) + st.tau * stage_dt(st);
}
__device__ __forceinline__ double tide_value(const Phys& ph, double t) {
  if (ph.tide_period <= 0.0) return ph.tide_amp;
  return ph.tide_amp * sin(2.0 * 3.14159265358979323846 * t / ph.tide_period + ph.tide_phase);
}

// Load all K modes of field f (base rows from the FP64 base state, higher rows
// from the group's correction array).
template <int K>
__device__ __forceinline__ void load_modes(T (&out)[K], const double* __restrict__ base, int64_t ne, int64_t e,
                                           const T* __restrict__ high, int64_t n, int64_t l, int f) {
#pragma unroll
  for (int i = 0; i < K; ++i) out[i] = i < 3 ? (T)base[(f * 3 + i) * ne + e] : high[(f * (K - 3) + (i - 3)) * n + l];
}

// ---------------------------------------------------------------------------
// auxiliary system of one order group:  M u = U, M v = V,
//   M[i][j] = (1/s) sum_{n < K(max deg)} H_n T[n][i][j],  H = xi + h_b.
// Solved as S u = s U with S = s M by an unpivoted LDL^T factorisation.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(128) k_usolve_corr(DevMesh m, int64_t g0, int64_t n, Phys ph,
                                                     const double* __restrict__ cb, const T* __restrict__ ch,
                                                     double* __restrict__ ub, T* __restrict__ uh,
                                                     unsigned* status) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int64_t e = g0 + l, ne = m.ne;
  constexpr int KH = K - 3, NP = K * (K + 1) / 2;
  T H[K];
  load_modes<K>(H, cb, ne, e, ch, n, l, 0);
  H[0] += (T)m.geo[G_HB0 * ne + e];
  H[1] += (T)m.geo[G_HB1 * ne + e];
  H[2] += (T)m.geo[G_HB2 * ne + e];
  const double sv = m.geo[G_S * ne + e];
  if (!((double)H[0] * cPhi0 / sv > ph.h_min)) atomicOr(status, (unsigned)ST_DEPTH);
  T A[NP];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int i = 0; i <= j; ++i) {
      T acc = 0;
#pragma unroll
      for (int nn = 0; nn < KMAX; ++nn)
        if (nn < ktr(i, j) && tnz(nn, i, j)) acc += H[nn] * cT[nn][pk(i, j)];
      A[pk(i, j)] = acc;
    }
  // LDL^T: A[pk(i,j)] (i > j) <- L_ij;  dg[j] = d_j, rd[j] = 1/d_j
  T dg[K], rd[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    T dj = A[pk(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) dj -= A[pk(j, k)] * A[pk(j, k)] * dg[k];
    dg[j] = dj;
    rd[j] = (T)1 / dj;
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      T w = A[pk(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) w -= A[pk(i, k)] * A[pk(j, k)] * dg[k];
      A[pk(i, j)] = w * rd[j];
    }
  }
  T x[2][K];
  load_modes<K>(x[0], cb, ne, e, ch, n, l, 1);
  load_modes<K>(x[1], cb, ne, e, ch, n, l, 2);
  const T s = (T)sv;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int k = 0; k < i; ++k) x[r][i] -= A[pk(i, k)] * x[r][k];
#pragma unroll
    for (int i = 0; i < K; ++i) x[r][i] *= rd[i];
#pragma unroll
    for (int i = K - 1; i >= 0; --i)
#pragma unroll
      for (int k = i + 1; k < K; ++k) x[r][i] -= A[pk(k, i)] * x[r][k];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const T v = x[r][i] * s;
      if (i < 3) ub[(r * 3 + i) * ne + e] = (double)v;
      else uh[(r * KH + (i - 3)) * n + l] = v;
    }
  }
}

template <int K>
static int usolve_group(cudaStream_t st, const DevMesh& m, const Groups& G, int p, const Phys& ph, StateDev c,
                        VelDev u, unsigned* status) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  k_usolve_corr<K><<<nblocks(n, 128), 128, 0, st>>>(m, g0, n, ph, c.cb, (const T*)c.ch[p], u.ub, (T*)u.uh[p],
                                                    status);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_usolve_corr(cudaStream_t st, const DevMesh& m, const Groups& G, const Phys& ph, StateDev c, VelDev u,
                       unsigned* status) {
  int r = usolve_group<6>(st, m, G, 2, ph, c, u, status);
  if (!r) r = usolve_group<10>(st, m, G, 3, ph, c, u, status);
  if (!r) r = usolve_group<15>(st, m, G, 4, ph, c, u, status);
  return r;
}

// ---------------------------------------------------------------------------
// correction edge flux.  Per side the traces are split into the P1 part (b)
// and the higher part (h).  With w = u.n, P = g xi (xi/2 + h_b):
//   A.n(b+h) - A.n(b) = ( U_h nx + V_h ny,
//                         U_h w + U_b w_h + g nx xi_h (xi_b + xi_h/2 + h_b),
//                         V_h w + V_b w_h + g ny xi_h (xi_b + xi_h/2 + h_b) )
// so the correction flux  F_h = 1/2 (A_h(L) + A_h(R) + lambda (c_h(L) - c_h(R)))
// carries no cancellation against the base flux.  F_f = F_b + F_h is the full
// LF flux for the test modes of degree >= 2.  Both are stored pre-weighted by
// |E| w_g at the points of the left element's direction.
// ---------------------------------------------------------------------------
struct Tr { T xb, Ub, Vb, ub, vb, xh, Uh, Vh, uh, vh; };

template <int PM>
__device__ __forceinline__ void side_traces(const DevMesh& m, const Groups& G, StateDev c, VelDev u, int64_t e,
                                            int k, bool reverse, Tr (&tr)[npts_for(PM)]) {
  constexpr int N = npts_for(PM), KM = Kof(PM), GI = PM - 2;
  const int64_t ne = m.ne;
  const int p = m.p[e], K = Kof(p);
  const T rs = (T)m.geo[G_RS * ne + e];
  int64_t l = 0, n = 1;
  const T* hc = nullptr;
  const T* hu = nullptr;
  if (p >= 2) {
    l = e - G.start[p]; n = G.start[p + 1] - G.start[p];
    hc = (const T*)c.ch[p]; hu = (const T*)u.uh[p];
  }
#pragma unroll
  for (int g = 0; g < N; ++g) tr[g] = Tr{0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < KM; ++i) {
    T cx, cU, cV, cu, cv;
    if (i < 3) {
      cx = (T)c.cb[(0 * 3 + i) * ne + e]; cU = (T)c.cb[(1 * 3 + i) * ne + e]; cV = (T)c.cb[(2 * 3 + i) * ne + e];
      cu = (T)u.ub[(0 * 3 + i) * ne + e]; cv = (T)u.ub[(1 * 3 + i) * ne + e];
    } else {
      if (i >= K) break;
      const int Kh = K - 3;
      cx = hc[(0 * Kh + i - 3) * n + l]; cU = hc[(1 * Kh + i - 3) * n + l]; cV = hc[(2 * Kh + i - 3) * n + l];
      cu = hu[(0 * Kh + i - 3) * n + l]; cv = hu[(1 * Kh + i - 3) * n + l];
    }
#pragma unroll
    for (int g = 0; g < N; ++g) {
      const T b = rs * (reverse ? cEB[GI][k][i][N - 1 - g] : cEB[GI][k][i][g]);
      if (i < 3) {
        tr[g].xb += cx * b; tr[g].Ub += cU * b; tr[g].Vb += cV * b; tr[g].ub += cu * b; tr[g].vb += cv * b;
      } else {
        tr[g].xh += cx * b; tr[g].Uh += cU * b; tr[g].Vh += cV * b; tr[g].uh += cu * b; tr[g].vh += cv * b;
      }
    }
  }
}

template <int PM>
__global__ void __launch_bounds__(128) k_edge_corr(DevMesh m, const int32_t* __restrict__ list, int64_t nl, Groups G,
                                                   Phys ph, Stage stg, StateDev c, VelDev u,
                                                   const double* __restrict__ lam_all, T* __restrict__ Fh,
                                                   T* __restrict__ Ff) {
  constexpr int N = npts_for(PM), GI = PM - 2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nl) return;
  const int64_t ed = list[idx], nE = m.nedge;
  const int L = m.eL[ed], R = m.eR[ed], info = m.einfo[ed];
  const int kL = info & 3, kR = (info >> 2) & 3, bc = info >> 4;
  const T len = (T)m.egeo[ed], nx = (T)m.egeo[nE + ed], ny = (T)m.egeo[2 * nE + ed];
  const T hA = (T)m.egeo[3 * nE + ed], hB = (T)m.egeo[4 * nE + ed];
  const T lam = (T)lam_all[ed];
  const T g = (T)ph.g;
  Tr a[N], b[N];
  side_traces<PM>(m, G, c, u, L, kL, false, a);
  if (R >= 0) {
    side_traces<PM>(m, G, c, u, R, kR, true, b);
  } else if (bc == 2) {
    const T xh = (T)tide_value(ph, stage_time(stg));
#pragma unroll
    for (int q = 0; q < N; ++q) { b[q] = a[q]; b[q].xb = xh; b[q].xh = 0; }
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const Tr& t = a[q];
      const T qb = t.Ub * nx + t.Vb * ny, qh = t.Uh * nx + t.Vh * ny;
      const T wb = t.ub * nx + t.vb * ny, wh = t.uh * nx + t.vh * ny;
      b[q] = Tr{t.xb, t.Ub - 2 * qb * nx, t.Vb - 2 * qb * ny, t.ub - 2 * wb * nx, t.vb - 2 * wb * ny,
                t.xh, t.Uh - 2 * qh * nx, t.Vh - 2 * qh * ny, t.uh - 2 * wh * nx, t.vh - 2 * wh * ny};
    }
  }
#pragma unroll
  for (int q = 0; q < N; ++q) {
    const T hb = hA + cES[GI][q] * (hB - hA);
    const Tr& x = a[q];
    const Tr& y = b[q];
    // base flux (P1 parts)
    const T wxb = x.ub * nx + x.vb * ny, wyb = y.ub * nx + y.vb * ny;
    const T pxb = g * x.xb * ((T)0.5 * x.xb + hb), pyb = g * y.xb * ((T)0.5 * y.xb + hb);
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
    Fh[(0 * N + q) * nl + idx] = wgt * Fh0;
    Fh[(1 * N + q) * nl + idx] = wgt * Fh1;
    Fh[(2 * N + q) * nl + idx] = wgt * Fh2;
    Ff[(0 * N + q) * nl + idx] = wgt * (Fb0 + Fh0);
    Ff[(1 * N + q) * nl + idx] = wgt * (Fb1 + Fh1);
    Ff[(2 * N + q) * nl + idx] = wgt * (Fb2 + Fh2);
  }
}

template <int PM>
static int edge_group(cudaStream_t st, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                      const Stage& stg, StateDev c, VelDev u, EdgeFlux fx) {
  const int64_t nl = ce.n[PM];
  if (nl == 0) return 0;
  k_edge_corr<PM><<<nblocks(nl, 128), 128, 0, st>>>(m, ce.list[PM], nl, G, ph, stg, c, u, fx.lam, (T*)fx.Fh[PM],
                                                    (T*)fx.Ff[PM]);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_edge_corr(cudaStream_t st, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                     const Stage& stg, StateDev c, VelDev u, EdgeFlux fx) {
  int r = edge_group<2>(st, m, ce, G, ph, stg, c, u, fx);
  if (!r) r = edge_group<3>(st, m, ce, G, ph, stg, c, u, fx);
  if (!r) r = edge_group<4>(st, m, ce, G, ph, stg, c, u, fx);
  return r;
}

// ---------------------------------------------------------------------------
// projection of one correction edge onto the test modes of an element:
//   r_f[q] -= sgn (1/s) sum_g F_g phihat_q(gamma_k(s_g))   (F_h for q < 3, F_f above).
// The base modes (q < 3) are accumulated in FP64 from the stored flux values,
// in the same point order on both sides of the edge, so that the mass
// exchanged through an edge cancels to FP64 round-off in every precision mode.
// ---------------------------------------------------------------------------
template <int PM, int KQ>
__device__ __forceinline__ void project_edge(T (&r)[3][KQ], double (&rb)[3][3], const EdgeFlux& fx,
                                             const CorrEdges& ce, int64_t sl, int k, bool right, double rs) {
  constexpr int N = npts_for(PM), GI = PM - 2;
  const int64_t nl = ce.n[PM];
  const T* Fh = (const T*)fx.Fh[PM];
  const T* Ff = (const T*)fx.Ff[PM];
  const double sg = right ? rs : -rs;
  const T sgt = (T)sg;
#pragma unroll
  for (int g = 0; g < N; ++g) {
    T fh[3], ff[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      fh[f] = Fh[(f * N + g) * nl + sl];
      if (KQ > 3) ff[f] = Ff[(f * N + g) * nl + sl];
    }
#pragma unroll
    for (int q = 0; q < 3 && q < KQ; ++q) {
      const double bq = sg * (right ? cEBd[GI][k][q][N - 1 - g] : cEBd[GI][k][q][g]);
#pragma unroll
      for (int f = 0; f < 3; ++f) rb[f][q] += (double)fh[f] * bq;
    }
#pragma unroll
    for (int q = 3; q < KQ; ++q) {
      const T bq = sgt * (right ? cEB[GI][k][q][N - 1 - g] : cEB[GI][k][q][g]);
#pragma unroll
      for (int f = 0; f < 3; ++f) r[f][q] += ff[f] * bq;
    }
  }
}

template <int KQ>
__device__ __forceinline__ void project_all_edges(T (&r)[3][KQ], double (&rb)[3][3], const DevMesh& m,
                                                  const EdgeFlux& fx, const CorrEdges& ce, int64_t e, double rs) {
  const int64_t ne = m.ne;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int ee = m.eedge[k * ne + e];
    const int64_t ed = ee >> 1;
    const bool right = ee & 1;
    const int cs = ce.slot[ed];
    if (cs < 0) continue;
    const int pm = cs >> 28;
    const int64_t sl = cs & 0x0fffffff;
    if (pm == 2) project_edge<2, KQ>(r, rb, fx, ce, sl, k, right, rs);
    else if (pm == 3) project_edge<3, KQ>(r, rb, fx, ce, sl, k, right, rs);
    else project_edge<4, KQ>(r, rb, fx, ce, sl, k, right, rs);
  }
}

// ---------------------------------------------------------------------------
// correction element update for one order group (K = K(p), p >= 2).
// Volume terms (Eq. 13 and its products) with J^{-1} folded into the
// contravariant coefficients  U^_i = (J^{-1} q_i)_xhat ..., u^_j, v^_j:
//   r_xi[q] += sum_i U^_i D_x[q][i] + V^_i D_y[q][i]
//   r_U[q]  += (1/s) [ sum_ij U_i (u^_j G_x[q][i][j] + v^_j G_y[q][i][j])
//                      + g (J^-1_xx P_x[q] + J^-1_yx P_y[q]) ]
//   r_V[q]  += (1/s) [ sum_ij V_i (...) + g (J^-1_xy P_x[q] + J^-1_yy P_y[q]) ]
//   P_k[q]   = sum_ij xi_i (xi_j/2 + hb_j) G_k[q][i][j]
// restricted to the non-base index triples, plus the source g grad h_b xi_q
// for q >= 3 and the correction edge projections.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(128) k_elem_corr(DevMesh m, CorrEdges ce, int64_t g0, int64_t n, Phys ph,
                                                   Stage stg, const double* __restrict__ cbS,
                                                   const T* __restrict__ chS, const T* __restrict__ chN,
                                                   T* __restrict__ chO, const double* __restrict__ ub,
                                                   const T* __restrict__ uh, EdgeFlux fx, double* __restrict__ rc) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int64_t e = g0 + l, ne = m.ne;
  constexpr int KH = K - 3;
  const double* geo = m.geo;
  T xi[K], U[K], V[K], uu[K], vv[K];
  load_modes<K>(xi, cbS, ne, e, chS, n, l, 0);
  load_modes<K>(U, cbS, ne, e, chS, n, l, 1);
  load_modes<K>(V, cbS, ne, e, chS, n, l, 2);
  load_modes<K>(uu, ub, ne, e, uh, n, l, 0);
  load_modes<K>(vv, ub, ne, e, uh, n, l, 1);
  const T rs = (T)geo[G_RS * ne + e];
  const T J0 = (T)geo[G_JI0 * ne + e], J1 = (T)geo[G_JI1 * ne + e];
  const T J2 = (T)geo[G_JI2 * ne + e], J3 = (T)geo[G_JI3 * ne + e];
  const T g = (T)ph.g;
  T hb[3] = {(T)geo[G_HB0 * ne + e], (T)geo[G_HB1 * ne + e], (T)geo[G_HB2 * ne + e]};
  T uc[K], vc[K], pp[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    uc[j] = J0 * uu[j] + J1 * vv[j];
    vc[j] = J2 * uu[j] + J3 * vv[j];
    pp[j] = (T)0.5 * xi[j] + (j < 3 ? hb[j] : (T)0);
  }
  T r[3][K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    T am = 0;
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (dnz(q, i) && !base2(q, i)) am += (J0 * U[i] + J1 * V[i]) * cD[0][q][i] + (J2 * U[i] + J3 * V[i]) * cD[1][q][i];
    T aU = 0, aV = 0, Px = 0, Py = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      T w = 0, px = 0, py = 0;
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (gnz(q, i, j) && !base3(q, i, j)) {
          const T gx = cG[0][q][pk(i, j)], gy = cG[1][q][pk(i, j)];
          w += uc[j] * gx + vc[j] * gy;
          px += pp[j] * gx;
          py += pp[j] * gy;
        }
      aU += U[i] * w; aV += V[i] * w;
      Px += xi[i] * px; Py += xi[i] * py;
    }
    r[0][q] = am;
    r[1][q] = rs * (aU + g * (J0 * Px + J2 * Py));
    r[2][q] = rs * (aV + g * (J1 * Px + J3 * Py));
    if (q >= 3) {
      r[1][q] += g * (T)geo[G_DHX * ne + e] * xi[q];
      r[2][q] += g * (T)geo[G_DHY * ne + e] * xi[q];
    }
  }
  double rb[3][3];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < 3; ++q) rb[f][q] = (double)r[f][q];
  project_all_edges<K>(r, rb, m, fx, ce, e, geo[G_RS * ne + e]);
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < 3; ++q) rc[(f * 3 + q) * ne + e] = rb[f][q];
  const T dt = (T)stage_dt(stg), a = (T)stg.a, b = (T)stg.b;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 3; q < K; ++q) {
      const int64_t ix = (f * KH + (q - 3)) * n + l;
      const T cs = f == 0 ? xi[q] : f == 1 ? U[q] : V[q];
      chO[ix] = stg.rhs_only ? r[f][q] : (stg.a != 0.0 ? a * chN[ix] : (T)0) + b * (cs + dt * r[f][q]);
    }
}

// p <= 1 elements with at least one correction edge: correction of the base modes only
__global__ void __launch_bounds__(128) k_elem_corr_lo(DevMesh m, CorrEdges ce, const int32_t* __restrict__ list,
                                                      int64_t nl, EdgeFlux fx, double* __restrict__ rc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nl) return;
  const int64_t e = list[idx], ne = m.ne;
  T r[3][3];
  double rb[3][3];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < 3; ++q) { r[f][q] = 0; rb[f][q] = 0.0; }
  project_all_edges<3>(r, rb, m, fx, ce, e, m.geo[G_RS * ne + e]);
  const int K = m.p[e] == 0 ? 1 : 3;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < 3; ++q) rc[(f * 3 + q) * ne + e] = q < K ? rb[f][q] : 0.0;
}

template <int K>
static int elem_group(cudaStream_t st, const DevMesh& m, const CorrEdges& ce, const Groups& G, int p, const Phys& ph,
                      const Stage& stg, StateDev cS, StateDev cN, StateDev cO, VelDev u, EdgeFlux fx, void* rc) {
  const int64_t g0 = G.start[p], n = G.start[p + 1] - g0;
  if (n == 0) return 0;
  k_elem_corr<K><<<nblocks(n, 128), 128, 0, st>>>(m, ce, g0, n, ph, stg, cS.cb, (const T*)cS.ch[p],
                                                  (const T*)cN.ch[p], (T*)cO.ch[p], u.ub, (const T*)u.uh[p], fx,
                                                  (double*)rc);
  count_launch();
  SWE_CUDA_OK(cudaGetLastError());
  return 0;
}

int launch_elem_corr(cudaStream_t st, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                     const Stage& stg, StateDev cS, StateDev cN, StateDev cO, VelDev u, EdgeFlux fx, void* rc,
                     const int32_t* edge_only, int64_t n_edge_only) {
  int r = elem_group<6>(st, m, ce, G, 2, ph, stg, cS, cN, cO, u, fx, rc);
  if (!r) r = elem_group<10>(st, m, ce, G, 3, ph, stg, cS, cN, cO, u, fx, rc);
  if (!r) r = elem_group<15>(st, m, ce, G, 4, ph, stg, cS, cN, cO, u, fx, rc);
  if (!r && n_edge_only > 0) {
    k_elem_corr_lo<<<nblocks(n_edge_only, 128), 128, 0, st>>>(m, ce, edge_only, n_edge_only, fx, (double*)rc);
    count_launch();
    SWE_CUDA_OK(cudaGetLastError());
  }
  return r;
}

}  // namespace CORR_NS
}  // namespace swedg
