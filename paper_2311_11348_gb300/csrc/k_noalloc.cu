// swe_rhs_p1_noalloc: the base right-hand side of an all-P1 mesh with no
// device allocation at all (the paper has no counterpart; see swedg.h).
//
// Some callers cannot allocate device memory: code that runs inside a
// region whose memory is budgeted up front (an embedding application that
// hands the solver fixed buffers and forbids cudaMalloc/cudaFree on its
// streams), or a host process that must not grow its device footprint after
// start-up.  For them the intermediate arrays of this one computation -- the
// auxiliary velocity u and the Lax-Friedrichs flux of every edge at its two
// Gauss points -- live in a file-scope __device__ array of fixed size,
// g_na_scratch, which every GPU that loads the library holds until the
// process exits.  The caller passes inputs and outputs; nothing else is
// allocated, by this file or by any library it calls.
//
// The same arithmetic as the context path (k_usolve_base, k_edge_base,
// k_elem_base): Sect. 2-3 of the paper for p = 1 with land walls.
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/swedg.h"
#include "common.h"
#include "kernels.h"
#include "tables.h"

namespace swedg {
namespace na {

constexpr int64_t NMAX = SWE_NOALLOC_MAX_ELEMENTS;
// per element: u [2][3] and edge flux [3 fields][2 points][3 local edges]
constexpr int64_t PER_ELEM = 6 + 18;
static __device__ __align__(256) double g_na_scratch[PER_ELEM * NMAX];

__constant__ double nB2[3][3][2];  // phihat_i(gamma_k(s_g)), i < 3, two-point rule
__constant__ double nW2[2], nS2[2];
__constant__ double nT1[3][3][3];  // T[n][i][j], n, i, j < 3
__constant__ double nLv[3][3];     // int lambda_v phihat_i
__constant__ double nGrad[3][2];   // grad phihat_q, q < 3
__constant__ double nPhi0;

// Set-up once per device context (with that device current): tables into
// constant memory and the device address of the scratch array.  The context
// is identified by its driver id, so a context re-created after
// cudaDeviceReset (whose constant memory starts zeroed) is set up again; a
// mutex serialises the set-up of host threads that call at the same time.
struct DevState {
  bool ready = false;
  unsigned long long ctx_id = 0;
  double* scratch = nullptr;
};
static DevState g_dev[64];
static std::mutex g_setup_mutex;

typedef CUresult (*PFN_ctxGetCurrent)(CUcontext*);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long*);

// driver id of the current context, 0 when there is none (or no driver entry)
static unsigned long long current_ctx_id() {
  static PFN_ctxGetCurrent get_current = nullptr;
  static PFN_ctxGetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = (PFN_ctxGetCurrent)f1;
      get_id = (PFN_ctxGetId)f2;
    }
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

static int setup(int dev, double** scratch) {
  if (dev < 0 || dev >= 64) return SWE_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long id0 = current_ctx_id();
  if (g_dev[dev].ready && id0 != 0 && id0 == g_dev[dev].ctx_id) {
    *scratch = g_dev[dev].scratch;
    return 0;
  }
  // the symbol lookup also makes the device's primary context current
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || p == nullptr) return SWE_ECUDA;
  const unsigned long long id = current_ctx_id();
  if (g_dev[dev].ready && id != 0 && id == g_dev[dev].ctx_id) {
    *scratch = g_dev[dev].scratch;
    return 0;
  }
  g_dev[dev].ready = false;
  const RefTables& R = tables();
  double B[3][3][2], T1[3][3][3], Lv[3][3], Gr[3][2];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int g = 0; g < 2; ++g) B[k][i][g] = R.EB[2][k][i][g];
  for (int n = 0; n < 3; ++n)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) T1[n][i][j] = R.T[n][i][j];
  std::memcpy(Lv, R.Lv, sizeof Lv);
  std::memcpy(Gr, R.grad1, sizeof Gr);
  if (cudaMemcpyToSymbol(nB2, B, sizeof B) != cudaSuccess ||
      cudaMemcpyToSymbol(nW2, R.ew[2], sizeof(double) * 2) != cudaSuccess ||
      cudaMemcpyToSymbol(nS2, R.es[2], sizeof(double) * 2) != cudaSuccess ||
      cudaMemcpyToSymbol(nT1, T1, sizeof T1) != cudaSuccess || cudaMemcpyToSymbol(nLv, Lv, sizeof Lv) != cudaSuccess ||
      cudaMemcpyToSymbol(nGrad, Gr, sizeof Gr) != cudaSuccess ||
      cudaMemcpyToSymbol(nPhi0, &R.phi0, sizeof(double)) != cudaSuccess)
    return SWE_ECUDA;
  g_dev[dev].scratch = (double*)p;
  g_dev[dev].ctx_id = id;
  g_dev[dev].ready = true;
  *scratch = (double*)p;
  return 0;
}

struct Geo {
  double rs, s, Ji[4];
};

__device__ __forceinline__ Geo element_geo(const double* __restrict__ xy, const int32_t* __restrict__ tri, int64_t e) {
  const int32_t v0 = tri[3 * e], v1 = tri[3 * e + 1], v2 = tri[3 * e + 2];
  const double x0 = xy[2 * v0], y0 = xy[2 * v0 + 1];
  const double J00 = xy[2 * v1] - x0, J01 = xy[2 * v2] - x0;
  const double J10 = xy[2 * v1 + 1] - y0, J11 = xy[2 * v2 + 1] - y0;
  const double det = J00 * J11 - J01 * J10;
  Geo G;
  G.s = sqrt(det);
  G.rs = 1.0 / G.s;
  G.Ji[0] = J11 / det; G.Ji[1] = -J01 / det; G.Ji[2] = -J10 / det; G.Ji[3] = J00 / det;
  return G;
}

__device__ __forceinline__ void hb_modes(const double* __restrict__ hv, const int32_t* __restrict__ tri, int64_t e,
                                         double s, double (&hb)[3]) {
  const double h[3] = {hv[tri[3 * e]], hv[tri[3 * e + 1]], hv[tri[3 * e + 2]]};
#pragma unroll
  for (int i = 0; i < 3; ++i) hb[i] = s * (h[0] * nLv[0][i] + h[1] * nLv[1][i] + h[2] * nLv[2][i]);
}

// An element is used only when its vertex ids lie in [0, nv) and it is
// counter-clockwise with positive area (det J_e > 0); any other element gets
// NaN rows and is a land edge to its neighbours.
__device__ __forceinline__ bool elem_ok(const double* __restrict__ xy, const int32_t* __restrict__ tri, int64_t nv,
                                        int64_t e) {
  const int32_t a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
  if (!(a >= 0 && b >= 0 && c >= 0 && a < nv && b < nv && c < nv)) return false;
  const double x0 = xy[2 * a], y0 = xy[2 * a + 1];
  const double det = (xy[2 * b] - x0) * (xy[2 * c + 1] - y0) - (xy[2 * c] - x0) * (xy[2 * b + 1] - y0);
  return det > 0.0;
}

// The element across local edge k of e, with e's local edge number kn in the
// neighbour's list, or -1 (land): a neighbour id outside [0, ne), an unusable
// neighbour, or one whose own list does not name e.  Both the edge and the
// element kernel decide through this one function, so every flux slot an
// element reads was written by the same call.
__device__ __forceinline__ int64_t mutual_nbr(const double* __restrict__ xy, const int32_t* __restrict__ tri,
                                              const int32_t* __restrict__ nbr, int64_t nv, int64_t ne, int64_t e,
                                              int k, int& kn) {
  const int64_t n = nbr[3 * e + k];
  if (n < 0 || n >= ne || n == e || !elem_ok(xy, tri, nv, n)) return -1;
  for (int j = 0; j < 3; ++j)
    if (nbr[3 * n + j] == e) { kn = j; return n; }
  return -1;
}

// auxiliary system of Sect. 3 for p = 1 (3 x 3, adjugate)
__global__ void k_na_usolve(int64_t nv, int64_t ne, const double* __restrict__ xy, const double* __restrict__ hv,
                            const int32_t* __restrict__ tri, const double* __restrict__ c, double* __restrict__ scr) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne || !elem_ok(xy, tri, nv, e)) return;
  const Geo G = element_geo(xy, tri, e);
  double hb[3];
  hb_modes(hv, tri, e, G.s, hb);
  double H[3], U[3], V[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) { H[i] = c[i * ne + e] + hb[i]; U[i] = c[(3 + i) * ne + e]; V[i] = c[(6 + i) * ne + e]; }
  const double a = H[0] * nT1[0][0][0];
  const double b = H[0] * nT1[0][0][1] + H[1] * nT1[1][0][1] + H[2] * nT1[2][0][1];
  const double cc = H[0] * nT1[0][0][2] + H[1] * nT1[1][0][2] + H[2] * nT1[2][0][2];
  const double d = H[0] * nT1[0][1][1] + H[1] * nT1[1][1][1] + H[2] * nT1[2][1][1];
  const double f = H[0] * nT1[0][1][2] + H[1] * nT1[1][1][2] + H[2] * nT1[2][1][2];
  const double h = H[0] * nT1[0][2][2] + H[1] * nT1[1][2][2] + H[2] * nT1[2][2][2];
  const double C00 = d * h - f * f, C01 = cc * f - b * h, C02 = b * f - cc * d;
  const double C11 = a * h - cc * cc, C12 = b * cc - a * f, C22 = a * d - b * b;
  const double r = G.s / (a * C00 + b * C01 + cc * C02);
  scr[0 * NMAX + e] = (C00 * U[0] + C01 * U[1] + C02 * U[2]) * r;
  scr[1 * NMAX + e] = (C01 * U[0] + C11 * U[1] + C12 * U[2]) * r;
  scr[2 * NMAX + e] = (C02 * U[0] + C12 * U[1] + C22 * U[2]) * r;
  scr[3 * NMAX + e] = (C00 * V[0] + C01 * V[1] + C02 * V[2]) * r;
  scr[4 * NMAX + e] = (C01 * V[0] + C11 * V[1] + C12 * V[2]) * r;
  scr[5 * NMAX + e] = (C02 * V[0] + C12 * V[1] + C22 * V[2]) * r;
}

// P1 traces of xi, U, V, u, v of element e on its local edge k at the two points
__device__ __forceinline__ void traces(const double* __restrict__ c, const double* __restrict__ scr, int64_t ne,
                                       int64_t e, int k, bool reverse, double rs, double (&t)[5][2]) {
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int gg = reverse ? 1 - g : g;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double coef = f < 3 ? c[(f * 3 + i) * ne + e] : scr[((f - 3) * 3 + i) * NMAX + e];
        acc += coef * nB2[k][i][gg];
      }
      t[f][g] = rs * acc;
    }
  }
}

// LF flux (Sect. 2) of every edge at its two Gauss points, stored once in the
// slot of its lower-numbered element, pre-weighted by |E| w_g / 2
__global__ void k_na_edge(int64_t nv, int64_t ne, const double* __restrict__ xy, const double* __restrict__ hv,
                          const int32_t* __restrict__ tri, const int32_t* __restrict__ nbr,
                          const double* __restrict__ c, double g, double* __restrict__ scr) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * ne) return;
  const int64_t e = t / 3;
  const int k = (int)(t % 3);
  if (!elem_ok(xy, tri, nv, e)) return;
  int kn = 0;
  const int64_t n = mutual_nbr(xy, tri, nbr, nv, ne, e, k, kn);
  if (n >= 0 && n < e) return;  // owned by the neighbour
  const int32_t va = tri[3 * e + (k + 1) % 3], vb = tri[3 * e + (k + 2) % 3];
  const double dx = xy[2 * vb] - xy[2 * va], dy = xy[2 * vb + 1] - xy[2 * va + 1];
  const double len = sqrt(dx * dx + dy * dy), nx = dy / len, ny = -dx / len;
  const double hA = hv[va], hB = hv[vb], hmid = 0.5 * (hA + hB);
  const Geo GL = element_geo(xy, tri, e);
  double a[5][2], b[5][2];
  traces(c, scr, ne, e, k, false, GL.rs, a);
  const double mL = nPhi0 * GL.rs;
  const double unL = (scr[0 * NMAX + e] * nx + scr[3 * NMAX + e] * ny) * mL;
  const double HL = c[e] * mL + hmid;
  double unR, HR;
  if (n >= 0) {
    const Geo GR = element_geo(xy, tri, n);
    traces(c, scr, ne, n, kn, true, GR.rs, b);
    const double mR = nPhi0 * GR.rs;
    unR = (scr[0 * NMAX + n] * nx + scr[3 * NMAX + n] * ny) * mR;
    HR = c[n] * mR + hmid;
  } else {  // land: mirror state
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double qn = a[1][q] * nx + a[2][q] * ny, wn = a[3][q] * nx + a[4][q] * ny;
      b[0][q] = a[0][q];
      b[1][q] = a[1][q] - 2.0 * qn * nx; b[2][q] = a[2][q] - 2.0 * qn * ny;
      b[3][q] = a[3][q] - 2.0 * wn * nx; b[4][q] = a[4][q] - 2.0 * wn * ny;
    }
    unR = -unL;
    HR = HL;
  }
  const double lam = fmax(fabs(unL), fabs(unR)) + fmax(sqrt(g * HL), sqrt(g * HR));
  double* F = scr + 6 * NMAX;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double hb = hA + nS2[q] * (hB - hA);
    const double wa = a[3][q] * nx + a[4][q] * ny, wb = b[3][q] * nx + b[4][q] * ny;
    const double pa = g * a[0][q] * (0.5 * a[0][q] + hb), pb = g * b[0][q] * (0.5 * b[0][q] + hb);
    const double F0 = (a[1][q] + b[1][q]) * nx + (a[2][q] + b[2][q]) * ny + lam * (a[0][q] - b[0][q]);
    const double F1 = a[1][q] * wa + b[1][q] * wb + (pa + pb) * nx + lam * (a[1][q] - b[1][q]);
    const double F2 = a[2][q] * wa + b[2][q] * wb + (pa + pb) * ny + lam * (a[2][q] - b[2][q]);
    const double wgt = 0.5 * len * nW2[q];
    F[((0 * 2 + q) * 3 + k) * NMAX + e] = wgt * F0;
    F[((1 * 2 + q) * 3 + k) * NMAX + e] = wgt * F1;
    F[((2 * 2 + q) * 3 + k) * NMAX + e] = wgt * F2;
  }
}

// volume, source and edge terms of the degree <= 1 test modes (closed form)
__global__ void k_na_elem(int64_t nv, int64_t ne, const double* __restrict__ xy, const double* __restrict__ hv,
                          const int32_t* __restrict__ tri, const int32_t* __restrict__ nbr,
                          const double* __restrict__ c, double g, const double* __restrict__ scr,
                          double* __restrict__ rhs) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  if (!elem_ok(xy, tri, nv, e)) {  // unusable element: NaN rows, nothing read
    for (int i = 0; i < 9; ++i) rhs[i * ne + e] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  const Geo G = element_geo(xy, tri, e);
  double hb[3];
  hb_modes(hv, tri, e, G.s, hb);
  double cc[3][3], u[2][3];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int i = 0; i < 3; ++i) cc[f][i] = c[(f * 3 + i) * ne + e];
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int i = 0; i < 3; ++i) u[f][i] = scr[(f * 3 + i) * NMAX + e];
  const int32_t v0 = tri[3 * e], v1 = tri[3 * e + 1], v2 = tri[3 * e + 2];
  const double dh1 = hv[v1] - hv[v0], dh2 = hv[v2] - hv[v0];
  const double dhx = dh1 * G.Ji[0] + dh2 * G.Ji[2], dhy = dh1 * G.Ji[1] + dh2 * G.Ji[3];
  double Axx = 0.0, Axy = 0.0, Ayx = 0.0, Ayy = 0.0, P = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Axx += cc[1][i] * u[0][i]; Axy += cc[1][i] * u[1][i];
    Ayx += cc[2][i] * u[0][i]; Ayy += cc[2][i] * u[1][i];
    P += cc[0][i] * (0.5 * cc[0][i] + hb[i]);
  }
  P *= g;
  const double m0 = G.s / nPhi0;
  double r[3][3];
  r[0][0] = 0.0;
  r[1][0] = g * dhx * cc[0][0];
  r[2][0] = g * dhy * cc[0][0];
#pragma unroll
  for (int q = 1; q < 3; ++q) {
    const double gx = G.rs * (nGrad[q][0] * G.Ji[0] + nGrad[q][1] * G.Ji[2]);
    const double gy = G.rs * (nGrad[q][0] * G.Ji[1] + nGrad[q][1] * G.Ji[3]);
    r[0][q] = (gx * cc[1][0] + gy * cc[2][0]) * m0;
    r[1][q] = gx * (Axx + P) + gy * Axy + g * dhx * cc[0][q];
    r[2][q] = gx * Ayx + gy * (Ayy + P) + g * dhy * cc[0][q];
  }
  const double* F = scr + 6 * NMAX;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int kn = 0;
    const int64_t n = mutual_nbr(xy, tri, nbr, nv, ne, e, k, kn);
    const bool right = n >= 0 && n < e;  // the flux is stored by the neighbour, in its direction
    const int64_t owner = right ? n : e;
    const int ko = right ? kn : k;
    const double sg = right ? G.rs : -G.rs;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double b0 = right ? nB2[k][q][1] : nB2[k][q][0];
      const double b1 = right ? nB2[k][q][0] : nB2[k][q][1];
#pragma unroll
      for (int f = 0; f < 3; ++f)
        r[f][q] += sg * (F[((f * 2 + 0) * 3 + ko) * NMAX + owner] * b0 + F[((f * 2 + 1) * 3 + ko) * NMAX + owner] * b1);
    }
  }
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < 3; ++q) rhs[(f * 3 + q) * ne + e] = r[f][q];
}

}  // namespace na
}  // namespace swedg

using namespace swedg;

extern "C" int swe_rhs_p1_noalloc(int64_t nv, const double* xy, const double* hv, int64_t ne, const int32_t* tri,
                                  const int32_t* nbr, const double* c, double g, double* rhs_out, void* stream) {
  if (ne < 1 || ne > na::NMAX || nv < 3 || !xy || !hv || !tri || !nbr || !c || !rhs_out || !(g > 0.0) ||
      !(g < INFINITY))
    return SWE_EINVAL;
  // an error left by earlier work on this thread is reported, not mistaken for ours later
  if (cudaGetLastError() != cudaSuccess) return SWE_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SWE_ECUDA;
  double* scr = nullptr;
  const int rc = na::setup(dev, &scr);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int T = 128;
  na::k_na_usolve<<<(unsigned)((ne + T - 1) / T), T, 0, s>>>(nv, ne, xy, hv, tri, c, scr);
  if (cudaGetLastError() != cudaSuccess) return SWE_ECUDA;
  na::k_na_edge<<<(unsigned)((3 * ne + T - 1) / T), T, 0, s>>>(nv, ne, xy, hv, tri, nbr, c, g, scr);
  if (cudaGetLastError() != cudaSuccess) return SWE_ECUDA;
  na::k_na_elem<<<(unsigned)((ne + T - 1) / T), T, 0, s>>>(nv, ne, xy, hv, tri, nbr, c, g, scr, rhs_out);
  return cudaGetLastError() == cudaSuccess ? 0 : SWE_ECUDA;
}
