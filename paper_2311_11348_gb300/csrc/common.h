// Internal declarations of libswedg shared by the host code and the kernels.
//
// Data layout in HBM (internal element order = caller's elements stably sorted
// by polynomial order p, so every order group is one contiguous range):
//   base state    cb[3 fields][3 modes][ne]            FP64   (modes of degree <= 1)
//   corr state    ch_p[3 fields][K(p)-3][n_p]  p = 2..4  FP64 or FP32
//   velocity      ub[2][3][ne] FP64,  uh_p[2][K(p)-3][n_p]
//   geometry      geo[NGEO][ne] FP64 (one row per quantity, coalesced)
//   edges         SoA arrays over interior edges first, then boundary edges
// All per-element arrays are structure-of-arrays so that consecutive threads
// (consecutive elements of one order group) issue coalesced 8-byte loads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>


namespace swedg {

constexpr int KMAX = 15;
constexpr int NB = 3;  // base modes: K(1)

__host__ __device__ constexpr int Kof(int p) { return (p + 1) * (p + 2) / 2; }
__host__ __device__ constexpr int deg_of(int i) { return i < 1 ? 0 : i < 3 ? 1 : i < 6 ? 2 : i < 10 ? 3 : 4; }
// Compile-time loop: f(IC<i>{}) for i in [B, E), so the index is a constant
// expression inside f (register arrays stay in registers and `if constexpr`
// removes the structural zeros of the reference tensors).
template <int N>
struct IC {
  static constexpr int value = N;
  __host__ __device__ constexpr operator int() const { return N; }
};
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    sfor<B + 1, E>(f);
  }
}

// Gauss-Legendre points per edge so that products of three traces of degree
// <= pmax (degree 3 pmax along the edge) are integrated exactly.
__host__ __device__ constexpr int npts_for(int pmax) { return pmax <= 1 ? 2 : (3 * pmax + 2) / 2; }

// rows of the per-element geometry table
enum {
  G_RS = 0,  // 1 / s_e, s_e = sqrt|det J_e|
  G_S,       // s_e
  G_JI0,     // d xhat / dx
  G_JI1,     // d xhat / dy
  G_JI2,     // d yhat / dx
  G_JI3,     // d yhat / dy
  G_GQ1X,    // grad phi_{e,2} (constant): x, y
  G_GQ1Y,
  G_GQ2X,    // grad phi_{e,3}
  G_GQ2Y,
  G_DHX,     // grad h_b
  G_DHY,
  G_HB0,     // modal h_b (P1 interpolant): 3 rows
  G_HB1,
  G_HB2,
  G_DIAM,    // inscribed diameter 4 |Omega_e| / perimeter
  G_GDHX,    // g grad h_b (source term of Eq. 5)
  G_GDHY,
  G_SQA,     // sqrt|Omega_e| = int phi_{e,1}
  G_M0,      // phihat_1 / s_e = sqrt 2 / s_e: the (constant) value of phi_{e,1}
  NGEO
};

// rows of the per-edge geometry table
enum {
  E_LEN = 0,  // |E|
  E_NX,       // outward unit normal of the left element
  E_NY,
  E_HA,       // h_b at gamma(0) and gamma(1) of the left element's parametrisation
  E_HB,
  E_HG0,      // h_b at the two Gauss points of the base rule
  E_HG1,
  E_HMID,     // h_b at the midpoint x_E (lambda, Eq. 10)
  E_WLEN,     // |E| w_g / 2 of the two-point rule (both weights are 1/2)
  E_NXW,      // E_WLEN * the normal: the base flux comes out pre-weighted
  E_NYW,
  NEGEO
};

// Per-stage SSP-RK combination  out = a * c^n + b * (c^(s) + dt * rhs),
// or out = rhs itself when rhs_only is set.
struct Stage {
  double a, b;
  int rhs_only;
  const double* dt;   // device array [members]: step of each ensemble member ...
  double dt_host;     // ... or this value for all members when dt == nullptr
  double t;           // time at the start of the step (host value, all members) ...
  const double* t_dev;  // ... or the device array [members] when non-null
  double tau;         // stage time = t_n + tau * dt
  int base_only;      // 1: the base part alone (no correction kernels, no rc)
};

struct Phys {
  double g, h_min;
  double tide_amp, tide_period, tide_phase;
  double fric_lin, fric_quad, f_c;  // bottom friction tau = fric_lin H + fric_quad |u| (means), Coriolis
  int src;                          // any of the three is nonzero
};

// Mesh topology and geometry on the device (internal order).
struct DevMesh {
  int64_t ne;
  int64_t nedge, nint;    // all edges, interior edges (boundary ones follow)
  const double* geo;      // [NGEO][ne]
  const int8_t* p;        // [ne]
  const int32_t* eedge;   // [3][ne]: (edge << 1) | side (side 1: the edge's right element)
  const int32_t* eL;      // [nedge] left element
  const int32_t* eR;      // [nedge] right element or -1
  const int32_t* einfo;   // [nedge] kL | kR << 2 | bc << 4   (bc: 0 interior, 1 land, 2 open sea)
  const double* egeo;     // [NEGEO][nedge] (rows E_*), in the left element's direction
  const float* geo32;     // FP32 copies of geo and egeo for the FP32 correction kernels
  const float* egeo32;
  const double* etb;      // [ne][3 local edges][4]: the degree-1 basis on the edge at the two
                          // points of the base rule, times 1/s_e: phi_{e,2}(g0), phi_{e,3}(g0),
                          // phi_{e,2}(g1), phi_{e,3}(g1) (points in the element's own direction)
  const int32_t* mem;     // [ne] ensemble member of each element (all 0 for a single mesh)
  const int32_t* emem;    // [nedge] member of each edge
  int32_t nmem;
  unsigned* mstatus;      // [nmem] status bits per member (ST_DEPTH, ST_NONFINITE), set beside the global word
};

// Correction edges grouped by pmax = max(p_L, p_R) in 2..4.
struct CorrEdges {
  int64_t n[5];           // per pmax
  const int32_t* list[5]; // edge ids
  const int32_t* slot;    // [nedge]: (pmax << 28) | slot within group, or -1
};

__device__ __forceinline__ double stage_dt(const Stage& st, int mem) { return st.dt ? st.dt[mem] : st.dt_host; }

// CFL bound of one element, d_e / ((|u_bar| + sqrt(g H_bar)) (2p+1)), in FP64
// from mode 0 of u and v and of the depth H = xi + h_b; an element mean is
// its mode 0 times sqrt 2 * rs (rs = 1 / sqrt(2 |Omega_e|)).  DBL_MAX where
// the bound is not a positive number (NaN never wins the minimum; the state
// checks report it).
__device__ __forceinline__ double cfl_bound(double u0, double v0, double H0, double rs, double g, double diam,
                                            int p) {
  const double r = 1.4142135623730951 * rs;
  const double ubar = u0 * r, vbar = v0 * r, Hbar = H0 * r;
  const double sp = sqrt(ubar * ubar + vbar * vbar) + sqrt(g * Hbar);
  const double dd = diam / (sp * (2.0 * p + 1.0));
  return (dd > 0.0 && dd < 1.7976931348623157e308) ? dd : 1.7976931348623157e308;
}

// min of d into dmin[mem] over the whole grid: positive doubles order like
// their bit patterns, so an integer atomicMin gives the exact minimum
// independent of the order of the blocks.  Every lane of the warp calls it
// (lanes without an element pass DBL_MAX); one atomic per warp when the
// warp's elements share a member (the usual case).
__device__ __forceinline__ void cfl_min_store(unsigned long long* dmin, int mem, double d) {
  const unsigned full = 0xffffffffu;
  const double dmax = 1.7976931348623157e308;
  const int mem0 = __shfl_sync(full, mem, 0);
  if (__all_sync(full, mem == mem0)) {
    for (int o = 16; o > 0; o >>= 1) d = fmin(d, __shfl_xor_sync(full, d, o));
    if ((threadIdx.x & 31) == 0 && d < dmax) atomicMin(dmin + mem0, (unsigned long long)__double_as_longlong(d));
  } else if (d < dmax) {
    atomicMin(dmin + mem, (unsigned long long)__double_as_longlong(d));
  }
}
__device__ __forceinline__ double stage_time(const Stage& st, int mem) {
  return (st.t_dev ? st.t_dev[mem] : st.t) + st.tau * stage_dt(st, mem);
}

}  // namespace swedg

#define SWE_CUDA_OK(call)                                      \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return ::swedg::cuda_fail(e__, #call, __FILE__, __LINE__); \
  } while (0)

namespace swedg {
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
}
