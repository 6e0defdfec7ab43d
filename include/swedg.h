/*
 * swedg.h -- C ABI of libswedg, a GB300 (sm_103a) solver for the quadrature-free,
 * p-adaptive discontinuous Galerkin discretisation of the 2D shallow water
 * equations of Faghih-Naini, Aizinger, Kuckuk, Angersbach and Koestler,
 * "p-adaptive discontinuous Galerkin method for the shallow water equations on
 * heterogeneous computing architectures" (2023).
 *
 * The problem statement the calls follow is Sect. 2: a triangulation with
 * bathymetry h_b, initial elevation xi and momentum q = (U, V), land
 * (q.n = 0) and open-sea (xi = xi_hat) boundaries, per-element polynomial
 * orders, and the semi-discrete system of Eqs. (8)-(9) advanced by an SSP
 * Runge-Kutta method.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns 0 on success or one of the negative SWE_E* codes; the
 *    text of the last failure is available from swe_last_error().
 *  - The library owns all device memory.  Buffers passed in are copied before
 *    the call returns and not retained, except by the asynchronous transfers
 *    (swe_*_async: until swe_sync returns) and the caller's CUDA stream in
 *    the parameters, which the context uses for its lifetime.
 *  - Pointers marked "host or device" may point to host memory or to device
 *    memory of the context's device (detected with cudaPointerGetAttributes).
 *  - State arrays use the layout c[3][15][ne]: field (0 = xi, 1 = U, 2 = V),
 *    modal index i of the orthonormal Dubiner basis (hierarchical: degree 0,
 *    then degree 1, ... ; K(p) = 1, 3, 6, 10, 15 modes for p = 0..4, Sect. 2
 *    Eqs. (11)-(12)), element in the caller's order.  Rows i >= K(p_e) are
 *    ignored on input and written as zero on output.
 *  - Coefficients are those of the basis orthonormal on each physical element
 *    Omega_e, phi_{e,i} = phihat_i o F_e^{-1} / sqrt|det J_e|, so the element
 *    mean of a field is c_1 / sqrt|Omega_e|.
 *  - A context is not thread safe; calls on one context are serialised on its
 *    CUDA stream.
 */
#ifndef SWEDG_H
#define SWEDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define SWE_OK 0
#define SWE_EINVAL (-1)   /* invalid argument or call order                        */
#define SWE_EMESH (-2)    /* degenerate triangle, non-manifold edge, bad vertex id   */
#define SWE_EDEPTH (-3)   /* an element mean of H = h_b + xi fell to or below h_min  */
#define SWE_ENONFINITE (-4) /* a non-finite value appeared in the state or the rhs  */
#define SWE_ECUDA (-5)    /* a CUDA runtime call failed                             */
#define SWE_ETIMEOUT (-6) /* a bounded device-side wait gave up                     */

/* precision modes of the higher-order correction (Sect. 3 order separation):
 * the base part (modes of degree <= 1, the CFL reduction, the RK update of the
 * base modes) is FP64 in every mode. */
#define SWE_PREC_FP64 0       /* correction in FP64 as well                          */
#define SWE_PREC_MIXED_FP32 1 /* correction arithmetic and storage in FP32           */
#define SWE_PREC_MIXED_TF32 2 /* as MIXED_FP32, but the momentum volume terms of the
                               * correction (the G contractions of Eq. 13) run on the
                               * tensor cores: every FP32 operand split into two TF32
                               * parts, three partial products, FP32 accumulation   */

typedef struct swe_ctx swe_ctx; /* opaque */

typedef struct {
  double g;           /* gravitational acceleration (Eq. 2)                          */
  double cfl;         /* CFL factor of the automatic time step                       */
  double h_min;       /* depth floor: an element mean H <= h_min is an error (-3)    */
  int rk_order;       /* 2: two-stage SSP-RK (Heun), 3: three-stage SSP-RK            */
  int precision;      /* SWE_PREC_*                                                  */
  double tide_amp;    /* open-sea elevation xi_hat(t) = amp * sin(2 pi t / period    */
  double tide_period; /*   + phase); period <= 0 gives the constant xi_hat = amp     */
  double tide_phase;
  void* cuda_stream;  /* cudaStream_t to run on; NULL = a stream the library creates */
  /* source terms of Eq. (5) (zero by default): bottom friction -tau_bf u with
   * tau_bf = fric_lin H + fric_quad |u| evaluated from the element means of H
   * and u (Sect. 3; the paper's setups use fric_lin = 1e-4 and fric_quad =
   * 0.009), and Coriolis f_c (V, -U).  fric_* >= 0, f_c finite, else -1. */
  double fric_lin;
  double fric_quad;
  double f_c;
} swe_params;

/* Fill *p with defaults: g = 9.81, cfl = 0.1, h_min = 1e-8, rk_order = 2,
 * FP64, no tide, no friction or Coriolis, library stream. */
void swe_default_params(swe_params* p);

/* Create a context on the current CUDA device.  *out is set on success. */
int swe_create(swe_ctx** out, const swe_params* params);

/* Release every resource of the context (NULL is accepted).  Device buffers
 * come from one stream-ordered memory pool per device that the library keeps
 * for the process: a destroyed context's memory goes back to that pool (for
 * the next context to reuse, without mapping new memory or synchronising the
 * device), not released to the CUDA driver. */
void swe_destroy(swe_ctx* ctx);

/* Text of the last error of the context; with ctx NULL, of the calling
 * thread's last failed swe_create or swe_mesh_adjacency. */
const char* swe_last_error(const swe_ctx* ctx);

/* Triangulation (Sect. 2: Omega = union of triangles Omega_e).
 *   xy[nv][2]   vertex coordinates (host)
 *   tri[ne][3]  vertex indices (host); clockwise triangles are re-oriented
 *               internally, which keeps "edge k is opposite vertex k"
 *   bc_tag      host [ne][3] or NULL; entry k describes the edge opposite
 *               vertex k: 0 = interior, or land if no neighbour matches;
 *               1 = land (q.n = 0); 2 = open sea (xi = xi_hat).  NULL = every
 *               edge without a neighbour is land.
 * Errors: SWE_EINVAL for nv < 3, ne < 1, a NULL xy or tri, or a boundary tag
 * outside 0..2; SWE_EMESH for a zero-area triangle, an out-of-range vertex
 * index or an edge shared by more than two triangles.  After an error the
 * context holds no mesh (calls that need one return SWE_EINVAL) until a
 * successful swe_set_mesh.  Resets orders to p = 1, the bathymetry to zero and
 * the state to zero. */
int swe_set_mesh(swe_ctx* ctx, int64_t nv, const double* xy, int64_t ne, const int32_t* tri,
                 const int8_t* bc_tag);

/* The adjacency swe_set_mesh builds, on the host alone (no context, no
 * device): the same validation of xy[nv][2] and tri[ne][3], then
 *   nbr_out[ne][3]  the triangle across the edge opposite vertex k, -1 on the
 *                   boundary (host, required)
 *   nbk_out[ne][3]  that triangle's own local index of the shared edge, -1 on
 *                   the boundary (host, may be NULL)
 * in the caller's triangle and vertex numbering (a clockwise triangle keeps
 * its vertex order here).  ne < 2^31.  Errors as swe_set_mesh (SWE_EINVAL
 * also for a NULL nbr_out); the text is swe_last_error(NULL) on the calling
 * thread. */
int swe_mesh_adjacency(int64_t nv, const double* xy, int64_t ne, const int32_t* tri, int32_t* nbr_out,
                       int8_t* nbk_out);

/* Bathymetry h_b (Eq. 2: H = h_b + xi), depths > 0 below the datum, given at
 * the vertices (host [nv]); the library uses its continuous piecewise-linear
 * interpolant. */
int swe_set_bathymetry(swe_ctx* ctx, const double* hb_vertex);

/* Per-element polynomial orders p_e in 0..4 (host [ne], caller's element
 * order).  The basis is hierarchical (Sect. 2), so the current state is kept:
 * modes beyond the new K(p_e) are dropped, new modes start at zero. */
int swe_set_orders(swe_ctx* ctx, const int8_t* p);

/* Modal state c[3][15][ne] (host or device) and its time t. */
int swe_set_state(swe_ctx* ctx, const double* c, double t);

/* Copy the modal state out (host or device c_out[3][15][ne]); t_out may be NULL. */
int swe_get_state(swe_ctx* ctx, double* c_out, double* t_out);

/* The same state in the packed layout (the paper has no counterpart; it moves
 * only the modes each element's order has): element by element in the
 * caller's order, element u's 3 K(p_u) coefficients field-major (xi, then U,
 * then V; modes 0 .. K(p_u)-1 each), K(p) = (p+1)(p+2)/2.  swe_packed_size
 * gives the number of doubles (sum of 3 K(p_u)) for the current orders, or
 * a negative error code.  Host or device buffers; SWE_EINVAL for NULL. */
int64_t swe_packed_size(swe_ctx* ctx);
int swe_set_state_packed(swe_ctx* ctx, const double* c, double t);
int swe_get_state_packed(swe_ctx* ctx, double* c_out, double* t_out);

/* Asynchronous variants (the paper has no counterpart: they let a caller
 * overlap the host<->device copies of one step's state with the computation
 * of the previous step).  The three calls only enqueue work on the context's
 * streams and return; swe_sync waits for everything enqueued on the context
 * and reports the first error, including the depth and finiteness checks of
 * the steps run since the previous status read.
 *   swe_set_state_packed_async  state (packed layout) and time t of every
 *                               member from c, host or device
 *   swe_run_async               nsteps CFL steps (dt_fixed <= 0) or fixed
 *                               steps of dt_fixed, as swe_run
 *   swe_get_state_packed_async  the current state (packed layout) into c_out,
 *                               host or device
 * Host buffers are copied on a copy stream per direction through two staging
 * buffers each (4 x swe_packed_size doubles of device memory, allocated by the
 * first asynchronous call and counted by swe_memory_bytes); they overlap with
 * the steps only when pinned (cudaHostAlloc / cudaHostRegister).  A buffer
 * passed to swe_set_state_packed_async must not be modified, and one passed
 * to swe_get_state_packed_async not be read, before swe_sync returns.
 * Order changes (swe_set_orders, swe_adapt) and the other calls may be mixed
 * in; they synchronise as documented for each. */
int swe_set_state_packed_async(swe_ctx* ctx, const double* c, double t);
int swe_run_async(swe_ctx* ctx, int64_t nsteps, double dt_fixed);
int swe_get_state_packed_async(swe_ctx* ctx, double* c_out);
int swe_sync(swe_ctx* ctx);

/* Modal coefficients of the continuous piecewise-linear interpolant of vertex
 * values (host vals[nv]) -> host or device modes_out[3][ne] (modes 1..3).
 * This is how the bathymetry enters the scheme; it also gives P1 initial
 * states. */
int swe_p1_modes(swe_ctx* ctx, const double* vals, double* modes_out);

/* Semi-discrete right-hand side dc/dt of Eq. (8) (orthonormal basis, so the
 * mass matrix is the identity) for the state c_in at the context's time:
 * rhs_out[3][15][ne].  c_in and rhs_out may be host or device.  The
 * context's own state is not changed. */
int swe_rhs(swe_ctx* ctx, const double* c_in, double* rhs_out);

/* The two parts of the order separation (Sect. 3, Eq. 13 and the text after
 * it): base_out holds every term whose test index and coefficient indices are
 * all modes of degree <= 1; corr_out holds the rest.  base + corr = rhs. */
int swe_rhs_parts(swe_ctx* ctx, const double* c_in, double* base_out, double* corr_out);

/* One SSP Runge-Kutta step of the context state (Sect. 2).  dt > 0 is used as
 * given; dt <= 0 takes the CFL step
 *   dt = cfl * min_e d_e / ((|u_bar_e| + sqrt(g H_bar_e)) (2 p_e + 1)),
 * d_e the inscribed diameter, u_bar and H_bar element means.  dt_used may be
 * NULL.  Returns SWE_EDEPTH / SWE_ENONFINITE when the step produced such a
 * state (the state is then left as computed). */
int swe_rk_step(swe_ctx* ctx, double dt, double* dt_used);

/* nsteps CFL steps (dt_fixed <= 0) or fixed steps of dt_fixed; t_out (may be
 * NULL) receives the final time.  Checks the status word once at the end. */
int swe_run(swe_ctx* ctx, int64_t nsteps, double dt_fixed, double* t_out);

/* Batched ensemble.  The mesh of swe_set_mesh may be the disjoint union of
 * independent members (e.g. the vertex and triangle arrays of several meshes
 * concatenated); member (host [ne], caller order) names the member 0 ..
 * nmembers-1 of every element, and the two elements of an edge must belong
 * to the same member.  Every member then keeps its own CFL time step and its
 * own time, while each kernel of a stage is still one launch over all
 * members.  The state is kept; every member's time is set to the context
 * time (swe_get_state's t).  nmembers = 1 with member = NULL restores a
 * single member.  SWE_EINVAL for ids out of range or a shared edge across
 * members. */
int swe_set_members(swe_ctx* ctx, int32_t nmembers, const int32_t* member);

/* Times of the members (host [nmembers]); swe_get_member_times also returns
 * the last step of every member in dt_out (host [nmembers], or NULL).  The
 * single-member calls (swe_set_state, swe_get_state, swe_run, swe_rk_step)
 * set every member's time and report member 0. */
int swe_set_member_times(swe_ctx* ctx, const double* t);
int swe_get_member_times(swe_ctx* ctx, double* t_out, double* dt_out);

/* Status of every ensemble member (host [nmembers]): the SWE_STATUS_* bits
 * that the steps since the last call (or since the last state upload) set
 * for that member's elements -- a mean depth at or below h_min, a non-finite
 * value in its state.  The paper has no counterpart: it lets a caller that
 * runs independent simulations in one context (a serving loop) tell which of
 * them failed when swe_run reports SWE_EDEPTH or SWE_ENONFINITE.  The bits
 * come from the depth checks of the steps and from the state check that
 * swe_run, swe_rk_step and swe_sync make before they return.  Reading clears
 * them. */
#define SWE_STATUS_DEPTH 1u
#define SWE_STATUS_NONFINITE 2u
int swe_member_status(swe_ctx* ctx, uint32_t* status_out);

/* Device memory held by the context (bytes; its buffers in the library's
 * pool); a serving loop admits requests by this footprint. */
int swe_memory_bytes(swe_ctx* ctx, int64_t* bytes);

/* Dynamic p-adaptivity (Sect. 2, end, and Sect. 3: with a hierarchical basis
 * an order change only adds or removes terms).  The paper's indicator (JRL)
 * is defined in an earlier paper, not in this one; this library uses a
 * modal-decay indicator of the elevation,
 *   s_e = sum_{deg i = p_e} xi_i^2 / sum_{deg i >= 1} xi_i^2   (0 if p_e = 0),
 * and sets p_e + 1 if s_e > theta_up and p_e < p_max, p_e - 1 if
 * s_e < theta_down and p_e > p_min.  The state is kept hierarchically (as in
 * swe_set_orders).  n_changed (or NULL) receives the number of elements whose
 * order changed, orders_out (host [ne] or NULL) the new orders.
 * SWE_EINVAL unless 0 <= p_min <= p_max <= 4 and theta_down <= theta_up. */
int swe_adapt(swe_ctx* ctx, double theta_up, double theta_down, int p_min, int p_max, int64_t* n_changed,
              int8_t* orders_out);

/* swe_run with swe_adapt after every `every` steps (the paper's dynamically
 * p-adaptive runs adapt during the simulation, Sect. 5). */
int swe_run_adaptive(swe_ctx* ctx, int64_t nsteps, int64_t every, double dt_fixed, double theta_up,
                     double theta_down, int p_min, int p_max, double* t_out);

/* Diagnostics of the context state:
 *   mass   = int xi dx = sum_e sqrt|Omega_e| xi_e1
 *   energy = 1/2 g int xi^2 + 1/2 int q.u  (u from the auxiliary system) */
int swe_mass(swe_ctx* ctx, double* m);
int swe_energy(swe_ctx* ctx, double* e);

/* Reference tensors the library generated (by its own Gauss quadrature) for
 * the contractions of Eq. (13):
 *   D[2][15][15]      D_k[q][i]    = int_T phihat_i d_k phihat_q
 *   G[2][15][15][15]  G_k[q][i][j] = int_T phihat_i phihat_j d_k phihat_q
 *   T[15][15][15]     T[n][i][j]   = int_T phihat_n phihat_i phihat_j
 * on the reference triangle T = {x, y >= 0, x + y <= 1}.  Host pointers, any
 * may be NULL.  Needs no device. */
int swe_reference_tensors(double* D, double* G, double* T);

/* Trace table of the factored edge integrals: npts Gauss-Legendre points
 * s_g in (0,1) with weights w_g (summing to 1) and
 *   B[k][i][g] = phihat_i(gamma_k(s_g)),
 * gamma_0(s) = (1-s, s), gamma_1(s) = (0, 1-s), gamma_2(s) = (s, 0), i.e.
 * local edge k is opposite reference vertex k and runs counter-clockwise.
 * npts in 1..8; host pointers.  Needs no device. */
int swe_edge_table(int npts, double* s, double* w, double* B);

/* Shared-memory image of the constant tensor-core operand of the
 * SWE_PREC_MIXED_TF32 volume contraction for K = 6, 10 or 15 modes (the paper
 * has no counterpart: it is the GB300 layout of the G_k tensors of Eq. 13).
 * The contraction runs as GEMMs of per-element rows of 2 K values (the
 * velocities, or the pressure products, for k = x^ then y^) against one
 * operand B with 16 K rows and 32 columns:
 *   B[16 i + q][k K + j] = G_k[q][i][j]
 * (zero for q >= K, for columns >= 2 K, for the base triples q, i, j < 3 and
 * for structural zeros).  The image holds two parts one after the other, each
 * 16 K x 32 floats: part 0 = G rounded to the nearest TF32 value (10 mantissa
 * bits, ties away from zero), part 1 = G - part 0 rounded the same way, so
 * their sum equals G to within 2^-22 |G|.  (row r, column c) of a part is at
 * float offset (r / 8) * 256 + (r % 8) * 32 + ((c / 4) ^ (r % 8)) * 4 + c % 4
 * (rows of 128 bytes, 16-byte units XOR-swizzled by the row index).  Returns
 * the number of floats (out may be NULL to query it), or SWE_EINVAL for
 * another K or cap too small.  Host pointer; needs no device. */
int64_t swe_tc_operand_image(int K, float* out, int64_t cap);

/* Launch shapes (the paper has no counterpart: they tune the GPU kernels to
 * the mesh, orders and device).  shape[6]:
 *   [0] resident blocks per SM of the grid-stride base edge and element
 *       kernels, 0..32 (0: no cap, one block per base_threads units of work)
 *   [1] threads per block of those kernels, 32..128, a multiple of 32
 *   [2] threads per block of the base u-solve, 32..256, a multiple of 32
 *   [3] threads per block of the correction u-solve and edge kernels,
 *       32..128, a multiple of 32
 *   [4] schedule of the correction element kernel (FP64 and mixed modes;
 *       ignored in SWE_PREC_MIXED_TF32): 0 = its higher test modes run
 *       before the base element kernel, 1 = beside it (on the correction
 *       stream, joined at the end of the stage)
 *   [5] work distribution of the capped base grids ([0] > 0), 0..16:
 *       0 = equal grid-stride shares per block; c > 0 = dynamic tiles: a
 *       block takes c * [1] consecutive edges (elements) at a time from a
 *       ticket counter until none are left, so blocks that share their SM
 *       with the concurrent correction kernels take fewer tiles
 * Defaults {2, 128, 256, 128, 0, 2}.  Results do not depend on the shape (every
 * unit of work is computed by one thread in the same order).  SWE_EINVAL for
 * a shape out of range. */
int swe_get_launch_shape(swe_ctx* ctx, int32_t* shape);
int swe_set_launch_shape(swe_ctx* ctx, const int32_t* shape);

/* Autotuner: for candidate launch shapes (coordinate descent: blocks per SM
 * in {1,2,3,4,6,0}, then base threads {64,128}, u-solve threads {128,256},
 * correction threads {64,128}, schedule {0,1}, base tiles {0,1,2,4}), runs `steps` CFL steps of the context's own
 * mesh and state, times them with CUDA events on the context stream, keeps
 * the fastest shape and restores the state and member times.  shape_out[6]
 * and ms_out (time per step of the choice) may be NULL.  Needs the state to
 * stay valid for the trial steps (errors of swe_run are returned). */
int swe_autotune(swe_ctx* ctx, int steps, int32_t* shape_out, double* ms_out);

/* Self-test of the device-side failure path (the paper has no counterpart):
 * every device wait of the library is bounded and, when it runs out, sets a
 * status bit that the next status read turns into SWE_ETIMEOUT, leaving the
 * context usable.  This call launches one block that waits `spins` times
 * (1..2^20) on an mbarrier nothing arrives on, so it returns SWE_ETIMEOUT;
 * the state is untouched. */
int swe_selftest_wait(swe_ctx* ctx, int64_t spins);

/* Per-kernel-family timing (ms, CUDA events on the context stream around
 * each family) accumulated while swe_profile(ctx, 1) is on; swe_run then
 * launches the steps directly instead of replaying its CUDA graph.  Families:
 * usolve, dt, edge_base, edge_corr, elem_corr, elem_base, other, vol_tc (the
 * tensor-core volume contraction of SWE_PREC_MIXED_TF32), and a last
 * entry "kernels" whose launch count is every kernel the library launched
 * since the last swe_profile call (graph replays included).  names (static
 * strings), ms and launches receive up to n entries; returns the number of
 * entries.  swe_profile resets all counters. */
int swe_profile(swe_ctx* ctx, int enable);
int swe_profile_read(swe_ctx* ctx, int n, const char** names, double* ms, int64_t* launches);

/* Allocation-free right-hand side of an all-P1 mesh (the paper has no
 * counterpart; this is a service for callers that cannot allocate).
 *
 * The context calls above allocate device memory (swe_set_mesh sizes every
 * buffer to the mesh).  Some callers cannot call cudaMalloc: an application
 * that hands the solver fixed, pre-allocated device buffers because its
 * device memory is partitioned up front, or because an allocation would
 * synchronise the device in the middle of its own pipelined stream work.
 * This call allocates nothing.  It computes what swe_rhs computes for p = 1
 * on every element, with land walls on every edge without a neighbour and
 * no tide, from caller-owned device arrays:
 *   xy[nv][2]   vertex coordinates          hv[nv]  vertex depths h_b
 *   tri[ne][3]  counter-clockwise triangles (vertex ids < nv)
 *   nbr[ne][3]  element across the edge opposite vertex k, or -1 (land)
 *   c[3][3][ne] modes 1..3 of xi, U, V (the basis of the context layout)
 *   rhs_out[3][3][ne]  the right-hand side of those modes
 * The intermediate values -- the auxiliary velocity u and the flux of every
 * edge at its two Gauss points -- live in one file-scope __device__ array
 * sized for SWE_NOALLOC_MAX_ELEMENTS elements (24 doubles each, 12.6 MB),
 * which every GPU that loads the library holds until the process exits.
 * Errors: SWE_EINVAL for ne < 1, ne > SWE_NOALLOC_MAX_ELEMENTS, nv < 3,
 * g not in (0, inf) or a NULL array; SWE_ECUDA when a launch fails, or when
 * the calling thread already had a CUDA error pending on entry (it is
 * reported here instead of being taken for this call's later).
 * Invalid mesh data never leads to an out-of-range access:
 *  - an element with a vertex id outside [0, nv), or that is clockwise or
 *    degenerate (det J_e <= 0), gets NaN rows and is land to its neighbours;
 *  - an edge is interior only when the relation is mutual: nbr[e][k] = n
 *    with n in [0, ne), n usable, and e in n's own list; otherwise (an id
 *    outside [0, ne), a one-sided entry) the edge is land for e.
 * No depth or finiteness status is reported (there is no context to hold it).
 * The first call on a device context copies the reference tables to constant
 * memory and looks up the device address of the scratch array
 * (cudaMemcpyToSymbol, cudaGetSymbolAddress; no allocation); make that first
 * call before any stream capture.  The set-up is serialised across host
 * threads and repeated when the device's context is re-created (for
 * instance after cudaDeviceReset).  Every call shares the one scratch array
 * and leaves its contents behind; nothing in it needs to start at zero (each
 * call writes every entry it reads), but calls that overlap on the GPU --
 * different streams, or different host threads -- race on it, so the caller
 * must serialise them.  Asynchronous on `stream` (a cudaStream_t; NULL is
 * the legacy default stream). */
#define SWE_NOALLOC_MAX_ELEMENTS 65536
int swe_rhs_p1_noalloc(int64_t nv, const double* xy, const double* hv, int64_t ne, const int32_t* tri,
                       const int32_t* nbr, const double* c, double g, double* rhs_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
