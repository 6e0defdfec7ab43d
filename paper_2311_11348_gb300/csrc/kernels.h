// Launchers of the libswedg kernels (all asynchronous on the given stream).
#pragma once
#include "common.h"

namespace swedg {

// Device view of one modal state (base + correction parts) in internal order.
struct StateDev {
  double* cb;        // [3][3][ne]
  void* ch[5];       // per order p = 2..4: [3][K(p)-3][n_p] of the correction type
  float* cb32;       // FP32 copy of cb for the FP32 correction (nullptr in FP64 mode)
};

struct VelDev {
  double* ub;        // [2][3][ne]
  void* uh[5];       // per p = 2..4: [2][K(p)-3][n_p]
  float* ub32;       // FP32 copy of ub (FP32 correction mode only)
  // per p = 2..4, element by element, every mode i < K(p) of the stage's state
  // and velocity as the correction kernels read them: tr = [n_p][K][4]
  // (xi, U, V, u), trv = [n_p][K] (v); written by the correction velocity
  // solve, read by the correction edge kernel (one 16-byte and one 4-byte
  // load per mode instead of five scattered loads)
  void* tr[5];
  void* trv[5];
};

struct Groups {
  int64_t start[6];  // internal element ranges per order p: [start[p], start[p+1])
};

struct EdgeFlux {
  double* Fb;        // [3][2][nedge] base flux (weighted by |E| w_g) at the 2-point rule
  double* Fbc;       // [3][2][nedge] two-point equivalent of the correction flux's share of the
                     // base modes (zero on edges without a p >= 2 side)
  void* Pf[5];       // per element order p = 2..4: [3 local edges][3 fields][K(p)-3][n_p]: the full flux of
                     // each of the element's (correction) edges projected onto its higher test modes (q >= 3),
                     // written by the correction edge kernel, read contiguously by the element kernel
};

// The mesh in the caller's element order, independent of the orders: what
// the device regrouping (k_regroup.cu) builds the internal arrays from.
// Edges are fixed: left element = the lower caller index of the two,
// interior edges first; eedge_u[k][u] = (edge << 1) | side of caller element
// u's local edge k (side 1: u is the edge's right element).
struct MeshStatic {
  int64_t ne, nedge;
  const double* geo_u;     // [NGEO][ne]
  const double* etb_u;     // [ne][12]
  const int32_t* eedge_u;  // [3][ne]
  const int32_t* eLu;      // [nedge] caller index of the left element
  const int32_t* eRu;      // [nedge] caller index of the right element or -1
  const int32_t* mem_u;    // [ne] ensemble member
};
// what the regrouping writes (every pointer a device array of the context)
struct DevMeshOut {
  int32_t* perm;   // [ne] internal -> caller
  int32_t* inv;    // [ne] caller -> internal
  int8_t* p;       // [ne] orders, internal
  double* geo;     // [NGEO][ne] internal
  float* geo32;    // [NGEO][ne]
  double* etb;     // [ne][12]
  int32_t* mem;    // [ne]
  int32_t* eedge;  // [3][ne]
  int32_t* eL;     // [nedge] internal index of the left element
  int32_t* eR;     // [nedge] internal index of the right element or -1
  int32_t* slot;   // [nedge] (pmax << 28) | position in the correction group, or -1
  int32_t* lists;  // [3][nedge] correction edge ids per pmax = 2, 3, 4
  int64_t* off;    // [ne] packed caller layout offsets (caller order)
};
// scratch of the partitions (sizes from regroup_blocks of ne and nedge)
struct RegroupScratch {
  int32_t* ecnt;  // [be][5]
  int64_t* eoff;  // [be][5]
  int32_t* gcnt;  // [bg][3]
  int64_t* goff;  // [bg][3]
  int64_t* psum;  // [be]
  int64_t* poff;  // [be + 1]
  int64_t* info;  // [16]: order group starts [0..5], correction group starts [6..9], packed size [10]
};
int64_t regroup_blocks(int64_t n);
// the internal arrays for the orders p_user (device, caller order); the
// group sizes land in W.info (device), for the host to read
int launch_regroup(cudaStream_t s, const MeshStatic& S, const int8_t* p_user, DevMeshOut D, RegroupScratch W);

// every kernel launch of the library is counted (for launch accounting)
void count_launch(int n = 1);

// status bits set by kernels
enum { ST_DEPTH = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

// Launch shapes the autotuner chooses (per context; the launchers read the
// shape of the context whose API call is running).
struct LaunchShape {
  int base_bpsm;       // resident blocks per SM of the grid-stride base edge / element kernels (0: uncapped)
  int base_threads;    // threads per block of those kernels (32..128)
  int usolve_threads;  // threads per block of the base u-solve (32..256)
  int corr_threads;    // threads per block of the correction u-solve and edge kernels (32..128)
  int split;           // 1: the correction element kernel's higher test modes run beside the base
                       // element kernel instead of before it (FP64 and mixed modes)
  int base_chunk;      // schedule of the capped base grids: 0 = equal grid-stride shares, c > 0 =
                       // dynamic tiles of c * base_threads edges / elements taken from a ticket counter
};
const LaunchShape& launch_shape();

// base-path tables (host -> constant memory of the base kernels)
void upload_base_tables();
void set_sm_count(int n);

// off == nullptr: the caller layout c[3][15][ne]; else packed, element u's
// 3 K(p_u) values (field-major) from off[u]
int launch_from_user(cudaStream_t s, const DevMesh& m, const Groups& G, const int32_t* perm, const int64_t* off,
                     int corr_fp32, const double* cu, StateDev st);
int launch_to_user(cudaStream_t s, const DevMesh& m, const Groups& G, const int32_t* perm, const int64_t* off,
                   int corr_fp32, StateDev st, double* cu);
int launch_sub(cudaStream_t s, const double* a, const double* b, double* out, int64_t n);

// dmin (or nullptr): per member, the running minimum of the elements' CFL
// bounds (DBL_MAX bits before the first stage of a step), folded in by the
// velocity solves of that stage and read (and reset) by launch_advance_time
int launch_usolve_base(cudaStream_t s, const DevMesh& m, const Groups& G, const Phys& ph, const double* cb,
                       double* ub, float* ub32, unsigned* status, unsigned long long* dmin);
// work: two zero-initialised counters per kernel for the dynamic schedule
// (left at zero when the launch ends), used by one launch at a time
int launch_edge_base(cudaStream_t s, const DevMesh& m, const Phys& ph, const Stage& stg, const double* cb,
                     const double* ub, EdgeFlux fx, unsigned* work);
int launch_elem_base(cudaStream_t s, const DevMesh& m, const Groups& G, const Phys& ph, const Stage& stg,
                     const double* cbS, const double* cbN, double* cbO, float* cbO32, const double* ub, EdgeFlux fx,
                     const void* rc, unsigned* work);
int launch_advance_time(cudaStream_t s, double* t_dev, unsigned long long* dmin, double cfl,
                        double dt_fixed, double* dt_dev, int nmem);
int launch_reset_min(cudaStream_t s, unsigned long long* dmin, int nmem);
// p[0 .. n) = v (member times set on the stream, without a host copy)
int launch_fill(cudaStream_t s, double* p, double v, int n);
int launch_indicator(cudaStream_t s, const DevMesh& m, const Groups& G, const int32_t* perm, int corr_fp32,
                     StateDev st, double up, double down, int pmin, int pmax, int8_t* p_user);
int launch_check_state(cudaStream_t s, const DevMesh& m, const Groups& G, int corr_fp32, StateDev st,
                       unsigned* status);
// deterministic two-pass reductions: mass and energy of a state
int launch_mass(cudaStream_t s, const DevMesh& m, const double* cb, double* partial, int nblk, double* out);
int launch_energy(cudaStream_t s, const DevMesh& m, const Groups& G, int corr_fp32, const Phys& ph, StateDev c,
                  VelDev u, double* partial, int nblk, double* out);

// correction kernels, one namespace per arithmetic type (FP64 / FP32)
// Streams of the order groups p = 2, 3, 4 in the correction launchers: the
// groups are independent (disjoint elements, edges and outputs), so they may
// run concurrently; all three the same stream when serial.
struct GroupStreams {
  cudaStream_t s[3];
};

#define SWE_CORR_DECL(NS)                                                                                        \
  namespace NS {                                                                                                 \
  void upload_tables();                                                                                          \
  int launch_usolve_corr(GroupStreams gs, const DevMesh& m, const Groups& G, const Phys& ph, StateDev c, VelDev u, \
                         unsigned* status, unsigned long long* dmin, void* rc);                                  \
  int launch_edge_corr(GroupStreams gs, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,   \
                       const Stage& stg, StateDev c, VelDev u, EdgeFlux fx);                                      \
  int launch_elem_corr(GroupStreams gs, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,   \
                       const Stage& stg, StateDev cS, StateDev cN, StateDev cO, VelDev u, EdgeFlux fx, void* rc,  \
                       int part);                                                                                 \
  }
SWE_CORR_DECL(corr64)
SWE_CORR_DECL(corr32)

// FP32 correction whose momentum volume terms run on the tensor cores
// (k_corr_tc.cu): the same launchers as corr32, elem_corr reads the volume
// terms that launch_vol_tc wrote to vol[32][elements of order >= 2].
namespace corrtc {
void upload_tables();
int upload_tc_tables();
int launch_usolve_corr(GroupStreams gs, const DevMesh& m, const Groups& G, const Phys& ph, StateDev c, VelDev u,
                       unsigned* status, unsigned long long* dmin, void* rc);
int launch_edge_corr(GroupStreams gs, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                     const Stage& stg, StateDev c, VelDev u, EdgeFlux fx);
int launch_elem_corr(GroupStreams gs, const DevMesh& m, const CorrEdges& ce, const Groups& G, const Phys& ph,
                     const Stage& stg, StateDev cS, StateDev cN, StateDev cO, VelDev u, EdgeFlux fx, void* rc,
                     int part, const float* vol);
int launch_vol_tc(cudaStream_t st, const DevMesh& m, const Groups& G, const Phys& ph, StateDev c, VelDev u,
                  float* vol, unsigned* status);
// host: the shared-memory image of the B operands for K = 6, 10, 15 (floats written, or needed when out is NULL)
int64_t tc_operand_image(int K, float* out, int64_t cap);
// a bounded wait on an mbarrier that nothing arrives on: sets ST_TIMEOUT
int launch_wait_selftest(cudaStream_t st, int64_t spins, unsigned* status);
}  // namespace corrtc

}  // namespace swedg
