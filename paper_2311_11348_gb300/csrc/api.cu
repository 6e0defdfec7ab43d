// libswedg host side: the C ABI of include/swedg.h, mesh processing (the
// per-element and per-edge geometry kept between steps, Sect. 4), grouping of the elements by
// polynomial order, device buffers and the SSP Runge-Kutta driver.
//
// One RK stage (Sect. 2 time stepping, Sect. 3 order separation):
//   usolve(base) + usolve(correction)      uH = q on every element
//   [first stage of a CFL step: dt = cfl * min ...]
//   edge_base -> edge_corr                 LF fluxes at Gauss points
//   elem_corr -> elem_base                 volume/source/edge projections and
//                                          the SSP-RK combination
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/swedg.h"
#include "common.h"
#include "kernels.h"
#include "tables.h"

namespace swedg {
static thread_local std::string g_cuda_err;
static thread_local int64_t* g_launch_counter = nullptr;
static thread_local const LaunchShape* g_shape = nullptr;
static const LaunchShape kDefaultShape{2, 128, 256, 128, 0, 2};
void count_launch(int n) {
  if (g_launch_counter) *g_launch_counter += n;
}
const LaunchShape& launch_shape() { return g_shape ? *g_shape : kDefaultShape; }
int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what,
           file, line);
  g_cuda_err = buf;
  return SWE_ECUDA;
}
}  // namespace swedg

using namespace swedg;

namespace {

const char* kFamilies[] = {"usolve", "dt", "edge_base", "edge_corr", "elem_corr", "elem_base", "other", "vol_tc"};
enum { F_USOLVE, F_DT, F_EDGEB, F_EDGEC, F_ELEMC, F_ELEMB, F_OTHER, F_VOLTC, NFAM };

}  // namespace

struct swe_ctx {
  swe_params prm{};
  cudaStream_t stream = nullptr;   // the caller's (or our) stream: base branch and ordering
  cudaStream_t stream2 = nullptr;  // the correction branch runs here, concurrently with the base
  cudaStream_t sg[2] = {nullptr, nullptr};  // its order groups p = 3, 4 (p = 2 stays on stream2)
  cudaEvent_t ev_gf = nullptr, ev_gj[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_u1 = nullptr, ev_u2 = nullptr, ev_c = nullptr, ev_dt = nullptr, ev_c2 = nullptr;
  bool own_stream = false;
  // asynchronous packed transfers: one copy stream per direction, two staging
  // buffers per direction (allocated on first use), events that order them
  // against the compute stream
  cudaStream_t cin = nullptr, cout = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_conv[2] = {}, ev_oready[2] = {}, ev_d2h[2] = {};
  double* d_stage_in[2] = {nullptr, nullptr};
  double* d_stage_out[2] = {nullptr, nullptr};
  int in_slot = 0, out_slot = 0;
  int device = 0;
  std::string err;
  bool have_mesh = false;   // a valid host mesh (topology built)
  bool dirty = true;        // the device data lag the host description
  bool keep_valid = false;  // keep_c holds the state to restore after the next device build
  std::vector<double> keep_c;
  double keep_t = 0.0;
  bool corr32 = false;  // FP32 correction (both mixed modes)
  bool tc = false;      // momentum volume terms of the correction on the tensor cores
  // host mesh, caller's element order, oriented counter-clockwise
  int64_t nv = 0, ne = 0;
  std::vector<double> xy, hv;
  std::vector<int32_t> tri;
  std::vector<int8_t> tag, p_user;
  std::vector<int32_t> member_user;  // ensemble member of each element (caller order)
  int32_t nmem = 1;
  std::vector<int64_t> nb;
  std::vector<int8_t> nbk;
  // internal numbering: perm[internal] = caller index
  Groups G{};
  int64_t nedge = 0;
  // the mesh in caller order and what the device regrouping writes
  MeshStatic ms{};
  DevMeshOut dout{};
  RegroupScratch rw{};
  // capacities (bytes) of the buffers sized by the order groups
  size_t cap_ch[3][5] = {}, cap_uh[5] = {}, cap_tr[5] = {}, cap_trv[5] = {}, cap_pf[5] = {};
  size_t cap_rc = 0, cap_vol = 0;
  // device
  std::vector<std::pair<void*, size_t>> allocs;
  DevMesh dm{};
  CorrEdges ce{};
  int32_t* d_perm = nullptr;
  StateDev st[3]{};
  VelDev vel{};
  EdgeFlux fx{};
  void* rc = nullptr;
  float* vol = nullptr;  // tensor-core volume terms [32][elements of order >= 2]
  double* d_user = nullptr;
  double* d_user2 = nullptr;
  int64_t* d_off = nullptr;  // packed caller layout: offset of each caller element's 3 K(p) values
  int64_t packed_n = 0;      // doubles in the packed layout
  double* d_dt = nullptr;
  double* d_t = nullptr;
  unsigned long long* d_dmin = nullptr;
  unsigned* d_status = nullptr;
  unsigned* d_mstatus = nullptr;  // [nmem] status bits per ensemble member
  double* d_partial = nullptr;
  double* d_red = nullptr;
  int8_t* d_newp = nullptr;  // orders proposed by the adaptivity indicator (caller order)
  unsigned* d_work = nullptr;  // ticket counters of the dynamic base schedule: edge kernel [0,1], element kernel [2,3]
  int nred = 0;
  // profiling
  bool prof = false;
  struct Ev { int fam; cudaEvent_t a, b; };
  std::vector<Ev> evs;
  std::vector<cudaEvent_t> pool;
  double prof_ms[NFAM] = {};
  int64_t prof_n[NFAM] = {};
  // CUDA graph of one step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = -1.0;
  int64_t graph_launches = 0;
  bool use_graph = true;
  // kernel launches issued by the library (graph replays count their kernels)
  int64_t launches = 0;
  int64_t dev_bytes = 0;  // device memory held by the context
  LaunchShape shape = kDefaultShape;
};

// Route count_launch() of the kernel launchers to this context while an API
// call runs.
struct LaunchScope {
  LaunchScope(swe_ctx* c) {
    g_launch_counter = c ? &c->launches : nullptr;
    g_shape = c ? &c->shape : nullptr;
  }
  ~LaunchScope() { g_launch_counter = nullptr; g_shape = nullptr; }
};

static int fail(swe_ctx* c, int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

static int cuda_err(swe_ctx* c, int rc) {
  if (rc == SWE_ECUDA && c) c->err = g_cuda_err;
  return rc;
}

#define CK(call)                                                  \
  do {                                                            \
    int rc__ = (call);                                            \
    if (rc__) return cuda_err(ctx, rc__);                         \
  } while (0)
#define CU(call)                                                  \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) return cuda_err(ctx, cuda_fail(e__, #call, __FILE__, __LINE__)); \
  } while (0)

// errors of the calls without a context (swe_create, swe_mesh_adjacency), per thread
static thread_local const char* g_create_err = "";
static thread_local std::string g_create_err_s;

// ------------------------------------------------------------------ memory
// Device buffers come from one stream-ordered memory pool per device, shared
// by the contexts of the process, that keeps freed memory for reuse: building
// and dropping contexts (ensemble cohorts of a server) then neither maps new
// memory nor synchronises the device, as cudaMalloc / cudaFree would while
// other contexts' kernels run.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static int device_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return cuda_fail(cudaErrorInvalidDevice, "device_pool", __FILE__, __LINE__);
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps pr{};
    pr.allocType = cudaMemAllocationTypePinned;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &pr);
    if (e != cudaSuccess) { g_pool[dev] = nullptr; return cuda_fail(e, "cudaMemPoolCreate", __FILE__, __LINE__); }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
  }
  *out = g_pool[dev];
  return 0;
}

// every stream of the context idle (before buffers are returned to the pool)
static void sync_streams(swe_ctx* ctx) {
  for (cudaStream_t s : {ctx->stream, ctx->stream2, ctx->sg[0], ctx->sg[1], ctx->cin, ctx->cout})
    if (s) cudaStreamSynchronize(s);
}

static void free_all(swe_ctx* ctx) {
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
  if (!ctx->allocs.empty()) sync_streams(ctx);
  for (auto& a : ctx->allocs) cudaFreeAsync(a.first, ctx->stream);
  ctx->allocs.clear();
  ctx->dev_bytes = 0;
}

// a buffer in stream order on the context stream; work on the context's other
// streams is ordered after it by the events that fork them from that stream
template <typename P>
static int dalloc(swe_ctx* ctx, P** out, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool;
  int rc = device_pool(ctx->device, &pool);
  if (rc) return rc;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync", __FILE__, __LINE__);
  ctx->allocs.push_back({p, bytes});
  ctx->dev_bytes += (int64_t)bytes;
  *out = (P*)p;
  return 0;
}

static void dfree(swe_ctx* ctx, void* p) {
  for (size_t i = 0; i < ctx->allocs.size(); ++i)
    if (ctx->allocs[i].first == p) {
      sync_streams(ctx);
      cudaFreeAsync(p, ctx->stream);
      ctx->dev_bytes -= (int64_t)ctx->allocs[i].second;
      ctx->allocs.erase(ctx->allocs.begin() + (long)i);
      return;
    }
}

// *p holds at least `need` bytes: the first allocation is exact, a later
// growth takes a quarter more so that repeated order changes rarely
// reallocate.  The contents are not kept.
template <typename P>
static int ensure_buf(swe_ctx* ctx, P** p, size_t* cap, size_t need) {
  if (need == 0) need = 16;
  if (*p && need <= *cap) return 0;
  const size_t bytes = *p ? need + need / 4 : need;
  if (*p) dfree(ctx, (void*)*p);
  *p = nullptr;
  *cap = 0;
  int rc = dalloc(ctx, p, bytes);
  if (!rc) *cap = bytes;
  return rc;
}

template <typename V>
static int upload(swe_ctx* ctx, V** out, const std::vector<V>& h) {
  int rc = dalloc(ctx, out, h.size() * sizeof(V));
  if (rc) return rc;
  if (!h.empty()) {  // from pageable memory: the call returns once the source has been staged
    cudaError_t e = cudaMemcpyAsync(*out, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
  }
  return 0;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ profiling
static void prof_mark(swe_ctx* ctx, int fam, bool begin) {
  if (!ctx->prof) return;
  if (begin) {
    cudaEvent_t a, b;
    if (ctx->pool.size() >= 2) { a = ctx->pool.back(); ctx->pool.pop_back(); b = ctx->pool.back(); ctx->pool.pop_back(); }
    else { cudaEventCreate(&a); cudaEventCreate(&b); }
    cudaEventRecord(a, ctx->stream);
    ctx->evs.push_back({fam, a, b});
  } else {
    cudaEventRecord(ctx->evs.back().b, ctx->stream);
  }
}

static void prof_collect(swe_ctx* ctx) {
  if (ctx->evs.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& ev : ctx->evs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    ctx->prof_ms[ev.fam] += ms;
    ctx->prof_n[ev.fam] += 1;
    ctx->pool.push_back(ev.a);
    ctx->pool.push_back(ev.b);
  }
  ctx->evs.clear();
}

// A kernel family's launches: an NVTX range on the host timeline (for Nsight
// tools; free without one) and, while profiling, CUDA events on the stream.
struct ProfScope {
  swe_ctx* c; int f;
  ProfScope(swe_ctx* c_, int f_) : c(c_), f(f_) {
    nvtxRangePushA(kFamilies[f]);
    prof_mark(c, f, true);
  }
  ~ProfScope() {
    prof_mark(c, f, false);
    nvtxRangePop();
  }
};

// ------------------------------------------------------------------ mesh
// f(a, b) over [0, n) in contiguous chunks on up to 16 host threads: the
// mesh setup loops, independent per element, edge or vertex (each chunk
// writes its own range), so the result does not depend on the split.
template <typename F>
static void host_parallel(int64_t n, F&& f) {
  const int64_t min_chunk = 1 << 15;
  int64_t nt = std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 16);
  nt = std::min<int64_t>(nt, (n + min_chunk - 1) / min_chunk);
  if (nt <= 1) {
    if (n > 0) f((int64_t)0, n);
    return;
  }
  const int64_t per = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (int64_t t = 1; t < nt; ++t) {
    const int64_t a = t * per, b = std::min(n, a + per);
    if (a < b) th.emplace_back([&f, a, b] { f(a, b); });
  }
  f((int64_t)0, std::min(n, per));
  for (auto& x : th) x.join();
}

static int build_topology(swe_ctx* ctx) {
  // Edge k of triangle e joins vertices a, b (the two other than vertex k).
  // Every edge is filed under its lower vertex (a counting sort over vertex
  // ids: linear in the mesh size), and the two sides of an interior edge are
  // the two entries of one vertex's bucket with the same upper vertex.
  const int64_t ne = ctx->ne, nv = ctx->nv;
  ctx->nb.assign(3 * ne, -1);
  ctx->nbk.assign(3 * ne, -1);
  const int32_t* tri = ctx->tri.data();
  auto ends = [&](int64_t x, int32_t& lo, int32_t& hi) {
    const int64_t e = x / 3;
    const int k = (int)(x % 3);
    const int32_t a = tri[3 * e + (k + 1) % 3], b = tri[3 * e + (k + 2) % 3];
    lo = std::min(a, b);
    hi = std::max(a, b);
  };
  std::vector<int64_t> start(nv + 1, 0), ent(3 * ne);
  int32_t lo, hi;
  for (int64_t x = 0; x < 3 * ne; ++x) { ends(x, lo, hi); ++start[lo + 1]; }
  for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
  {
    std::vector<int64_t> cur(start.begin(), start.end() - 1);
    for (int64_t x = 0; x < 3 * ne; ++x) { ends(x, lo, hi); ent[cur[lo]++] = x; }
  }
  // pair within each bucket (a vertex's bucket is touched by its chunk only);
  // a chunk stops at its first bad vertex, and the lowest one is reported
  struct Bad { int64_t v, what; int kind; };  // kind 1: third triangle on (v, what); 2: triangle `what`
  std::vector<Bad> bad;
  std::mutex mu;
  host_parallel(nv, [&](int64_t v0, int64_t v1) {
    int32_t lo_, hi_, hx;
    for (int64_t v = v0; v < v1; ++v)
      for (int64_t i = start[v]; i < start[v + 1]; ++i) {
        const int64_t x = ent[i];
        if (x < 0) continue;  // the second side of an edge already paired
        ends(x, lo_, hx);
        int64_t match = -1;
        for (int64_t j = i + 1; j < start[v + 1]; ++j) {
          const int64_t y = ent[j];
          if (y < 0) continue;
          ends(y, lo_, hi_);
          if (hi_ != hx) continue;
          if (match >= 0) {
            std::lock_guard<std::mutex> g(mu);
            bad.push_back({v, hx, 1});
            return;
          }
          match = j;
        }
        if (match < 0) continue;  // boundary edge
        const int64_t y = ent[match];
        const int64_t A = x / 3, B = y / 3;
        if (A == B) {
          std::lock_guard<std::mutex> g(mu);
          bad.push_back({v, A, 2});
          return;
        }
        ctx->nb[x] = B; ctx->nbk[x] = (int8_t)(y % 3);
        ctx->nb[y] = A; ctx->nbk[y] = (int8_t)(x % 3);
        ent[match] = -1;
      }
  });
  if (!bad.empty()) {
    const Bad b = *std::min_element(bad.begin(), bad.end(), [](const Bad& p, const Bad& q) { return p.v < q.v; });
    if (b.kind == 1)
      return fail(ctx, SWE_EMESH, "edge (%lld,%lld) is shared by more than 2 triangles", (long long)b.v,
                  (long long)b.what);
    return fail(ctx, SWE_EMESH, "triangle %lld repeats a vertex", (long long)b.what);
  }
  return 0;
}

// Buffers whose sizes follow the order groups (the current G and ce.n): the
// correction parts of the three RK states, of the velocity and of the trace
// records, the correction edges' projections, rc, the tensor-core volume
// terms and the per-element correction edge slots.  Grown as needed (a new
// buffer starts zeroed; the contents of a regrown one are not kept).
static int alloc_group_buffers(swe_ctx* ctx) {
  const size_t ts = ctx->corr32 ? sizeof(float) : sizeof(double);
  auto grow = [&](auto** ptr, size_t* cap, size_t need) -> int {
    void* before = (void*)*ptr;
    int rc = ensure_buf(ctx, ptr, cap, need);
    // zeroed on the context stream, ahead of the kernels that fill it
    if (!rc && (void*)*ptr != before)
      rc = cudaMemsetAsync((void*)*ptr, 0, *cap, ctx->stream) == cudaSuccess ? 0 : SWE_ECUDA;
    return rc;
  };
  int rc = 0;
  for (int p = 2; p < 5 && !rc; ++p) {
    const size_t n = (size_t)(ctx->G.start[p + 1] - ctx->G.start[p]), K = (size_t)Kof(p);
    for (int s = 0; s < 3 && !rc; ++s) rc = grow(&ctx->st[s].ch[p], &ctx->cap_ch[s][p], ts * 3 * (K - 3) * n);
    if (!rc) rc = grow(&ctx->vel.uh[p], &ctx->cap_uh[p], ts * 2 * (K - 3) * n);
    if (!rc) rc = grow(&ctx->vel.tr[p], &ctx->cap_tr[p], ts * 4 * K * n);
    if (!rc) rc = grow(&ctx->vel.trv[p], &ctx->cap_trv[p], ts * K * n);
    if (!rc) rc = grow(&ctx->fx.Pf[p], &ctx->cap_pf[p], ts * 3 * 3 * (K - 3) * n);
  }
  const size_t nrc = (size_t)std::max<int64_t>(ctx->ne - ctx->G.start[2], 1);
  if (!rc) rc = grow(&ctx->rc, &ctx->cap_rc, sizeof(double) * 4 * nrc);
  if (!rc && ctx->tc) rc = grow(&ctx->vol, &ctx->cap_vol, sizeof(float) * 32 * nrc);
  return rc ? cuda_err(ctx, rc) : 0;
}

// Group the elements for the orders in d_newp (caller order) on the device:
// the internal arrays, the group sizes (read back: one small copy and a
// stream synchronisation) and the buffers that follow them.  keep_state
// carries the state over hierarchically through the caller layout (modes
// beyond an element's new order dropped, new modes zero).
static int regroup(swe_ctx* ctx, bool keep_state) {
  nvtxRangePushA("regroup");
  const int64_t packed_before = ctx->packed_n;
  if (keep_state)  // the state in the old internal order, out to the caller layout
    CK(launch_to_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, nullptr, ctx->corr32, ctx->st[0], ctx->d_user));
  CK(launch_regroup(ctx->stream, ctx->ms, ctx->d_newp, ctx->dout, ctx->rw));
  int64_t info[11] = {};
  CU(cudaMemcpyAsync(info, ctx->rw.info, sizeof info, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  for (int p = 0; p <= 5; ++p) ctx->G.start[p] = info[p];
  for (int pm = 0; pm < 5; ++pm) ctx->ce.n[pm] = (pm >= 2 && ctx->nedge > 0) ? info[6 + pm - 1] - info[6 + pm - 2] : 0;
  ctx->packed_n = info[10];
  CK(alloc_group_buffers(ctx));
  // edges that no longer touch a p >= 2 element carry no correction flux
  CU(cudaMemsetAsync(ctx->fx.Fbc, 0, sizeof(double) * 6 * (size_t)std::max<int64_t>(ctx->nedge, 1), ctx->stream));
  if (keep_state)
    CK(launch_from_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, nullptr, ctx->corr32, ctx->d_user, ctx->st[0]));
  if (ctx->packed_n != packed_before)  // the asynchronous staging buffers follow the packed size
    for (int k = 0; k < 2; ++k) {
      if (ctx->d_stage_in[k]) { CU(cudaStreamSynchronize(ctx->cin)); dfree(ctx, ctx->d_stage_in[k]); }
      if (ctx->d_stage_out[k]) { CU(cudaStreamSynchronize(ctx->cout)); dfree(ctx, ctx->d_stage_out[k]); }
      ctx->d_stage_in[k] = ctx->d_stage_out[k] = nullptr;
    }
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }  // sizes and grids changed
  nvtxRangePop();
  return 0;
}

// Build the mesh data in the caller's order on the host (geometry, edges),
// the fixed-size device buffers, and the order-dependent ones through the
// device regrouping; the state is reset to zero (callers that keep it go
// through the caller layout).
static int build_device(swe_ctx* ctx) {
  free_all(ctx);
  for (int k = 0; k < 2; ++k) ctx->d_stage_in[k] = ctx->d_stage_out[k] = nullptr;  // freed with the rest
  for (int s = 0; s < 3; ++s)
    for (int p = 0; p < 5; ++p) { ctx->st[s].ch[p] = nullptr; ctx->cap_ch[s][p] = 0; }
  for (int p = 0; p < 5; ++p) {
    ctx->vel.uh[p] = ctx->vel.tr[p] = ctx->vel.trv[p] = nullptr;
    ctx->fx.Pf[p] = nullptr;
    ctx->cap_uh[p] = ctx->cap_tr[p] = ctx->cap_trv[p] = ctx->cap_pf[p] = 0;
  }
  ctx->rc = nullptr; ctx->vol = nullptr; ctx->cap_rc = ctx->cap_vol = 0;
  std::memset(&ctx->ce, 0, sizeof ctx->ce);
  const int64_t ne = ctx->ne;
  const RefTables& R = tables();
  // geometry, caller order
  std::vector<double> geo((size_t)NGEO * ne);
  host_parallel(ne, [&](int64_t u0, int64_t u1) {
  for (int64_t u = u0; u < u1; ++u) {
    const int32_t* v = &ctx->tri[3 * u];
    const double x0 = ctx->xy[2 * v[0]], y0 = ctx->xy[2 * v[0] + 1];
    const double J00 = ctx->xy[2 * v[1]] - x0, J01 = ctx->xy[2 * v[2]] - x0;
    const double J10 = ctx->xy[2 * v[1] + 1] - y0, J11 = ctx->xy[2 * v[2] + 1] - y0;
    const double det = J00 * J11 - J01 * J10;
    const double sq = std::sqrt(det), rs = 1.0 / sq;
    const double Ji[4] = {J11 / det, -J01 / det, -J10 / det, J00 / det};
    auto G_ = [&](int row) -> double& { return geo[(size_t)row * ne + u]; };
    G_(G_RS) = rs; G_(G_S) = sq;
    G_(G_JI0) = Ji[0]; G_(G_JI1) = Ji[1]; G_(G_JI2) = Ji[2]; G_(G_JI3) = Ji[3];
    for (int q = 1; q < 3; ++q) {
      const double gx = rs * (R.grad1[q][0] * Ji[0] + R.grad1[q][1] * Ji[2]);
      const double gy = rs * (R.grad1[q][0] * Ji[1] + R.grad1[q][1] * Ji[3]);
      G_(q == 1 ? G_GQ1X : G_GQ2X) = gx;
      G_(q == 1 ? G_GQ1Y : G_GQ2Y) = gy;
    }
    const double h0 = ctx->hv[v[0]], h1 = ctx->hv[v[1]], h2 = ctx->hv[v[2]];
    G_(G_DHX) = (h1 - h0) * Ji[0] + (h2 - h0) * Ji[2];
    G_(G_DHY) = (h1 - h0) * Ji[1] + (h2 - h0) * Ji[3];
    const double hvv[3] = {h0, h1, h2};
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int w = 0; w < 3; ++w) acc += hvv[w] * R.Lv[w][i];
      G_(G_HB0 + i) = sq * acc;
    }
    double per = 0.0;
    for (int k = 0; k < 3; ++k) {
      const int32_t a = v[(k + 1) % 3], b = v[(k + 2) % 3];
      per += std::hypot(ctx->xy[2 * b] - ctx->xy[2 * a], ctx->xy[2 * b + 1] - ctx->xy[2 * a + 1]);
    }
    G_(G_DIAM) = 2.0 * det / per;
    G_(G_GDHX) = ctx->prm.g * G_(G_DHX);
    G_(G_GDHY) = ctx->prm.g * G_(G_DHY);
    G_(G_SQA) = std::sqrt(0.5 * det);
    G_(G_M0) = R.phi0 * rs;
  }
  });
  std::vector<double> etb((size_t)12 * ne);
  host_parallel(ne, [&](int64_t u0, int64_t u1) {
    for (int64_t u = u0; u < u1; ++u)
      for (int k = 0; k < 3; ++k) {
        const double rs = geo[(size_t)G_RS * ne + u];
        double* t = &etb[(size_t)(3 * u + k) * 4];
        t[0] = rs * R.EB[2][k][1][0]; t[1] = rs * R.EB[2][k][2][0];
        t[2] = rs * R.EB[2][k][1][1]; t[3] = rs * R.EB[2][k][2][1];
      }
  });
  // edges: left element = the lower caller index, interior edges first, then
  // the boundary edges, each part sorted by the left element (an edge is made
  // by its lower element; counts per element place it without a sort)
  struct E { int32_t L, R, info; double len, nx, ny, hA, hB; };
  std::vector<int64_t> offI(ne + 1, 0), offB(ne + 1, 0);
  host_parallel(ne, [&](int64_t u0, int64_t u1) {
    for (int64_t u = u0; u < u1; ++u) {
      int ci = 0, cb = 0;
      for (int k = 0; k < 3; ++k) {
        const int64_t n = ctx->nb[3 * u + k];
        if (n < 0) ++cb;
        else if (n > u) ++ci;
      }
      offI[u + 1] = ci;
      offB[u + 1] = cb;
    }
  });
  for (int64_t u = 0; u < ne; ++u) { offI[u + 1] += offI[u]; offB[u + 1] += offB[u]; }
  const int64_t nI = offI[ne];
  std::vector<E> ed((size_t)(nI + offB[ne]));
  host_parallel(ne, [&](int64_t u0, int64_t u1) {
    for (int64_t u = u0; u < u1; ++u) {
      int64_t pi = offI[u], pb = nI + offB[u];
      for (int k = 0; k < 3; ++k) {
        const int64_t n = ctx->nb[3 * u + k];
        if (n >= 0 && n < u) continue;  // made by the other side
        E x;
        int32_t Rr = -1, kR = 0, bc;
        if (n >= 0) {
          bc = 0;
          Rr = (int32_t)n; kR = ctx->nbk[3 * u + k];
        } else {
          bc = ctx->tag[3 * u + k] == 2 ? 2 : 1;
        }
        x.L = (int32_t)u; x.R = Rr;
        x.info = k | (kR << 2) | (bc << 4);
        const int32_t a = ctx->tri[3 * u + (k + 1) % 3], b = ctx->tri[3 * u + (k + 2) % 3];
        const double dx = ctx->xy[2 * b] - ctx->xy[2 * a], dy = ctx->xy[2 * b + 1] - ctx->xy[2 * a + 1];
        x.len = std::hypot(dx, dy);
        x.nx = dy / x.len; x.ny = -dx / x.len;
        x.hA = ctx->hv[a]; x.hB = ctx->hv[b];
        ed[(size_t)(n >= 0 ? pi++ : pb++)] = x;
      }
    }
  });
  const int64_t nE = (int64_t)ed.size();
  ctx->nedge = nE;
  if (nE >= (1ll << 27) || ne >= (1ll << 30)) return fail(ctx, SWE_EINVAL, "mesh too large for 27-bit edge slots");
  std::vector<int32_t> eLu(nE), eRu(nE), einfo(nE), eedge_u(3 * ne, -1), emem(nE);
  std::vector<double> egeo((size_t)NEGEO * nE);
  const int64_t nint = nI;
  host_parallel(nE, [&](int64_t i0, int64_t i1) {
  for (int64_t i = i0; i < i1; ++i) {
    eLu[i] = ed[i].L; eRu[i] = ed[i].R; einfo[i] = ed[i].info;
    emem[i] = ctx->member_user[ed[i].L];
    auto E_ = [&](int row) -> double& { return egeo[(size_t)row * nE + i]; };
    E_(E_LEN) = ed[i].len; E_(E_NX) = ed[i].nx; E_(E_NY) = ed[i].ny;
    E_(E_HA) = ed[i].hA; E_(E_HB) = ed[i].hB;
    E_(E_HG0) = ed[i].hA + R.es[2][0] * (ed[i].hB - ed[i].hA);
    E_(E_HG1) = ed[i].hA + R.es[2][1] * (ed[i].hB - ed[i].hA);
    E_(E_HMID) = 0.5 * (ed[i].hA + ed[i].hB);
    E_(E_WLEN) = 0.5 * ed[i].len * R.ew[2][0];  // the two weights of the base rule are equal
    E_(E_NXW) = E_(E_WLEN) * ed[i].nx;
    E_(E_NYW) = E_(E_WLEN) * ed[i].ny;
    eedge_u[(size_t)(ed[i].info & 3) * ne + ed[i].L] = (int32_t)(i << 1);
    if (ed[i].R >= 0) eedge_u[(size_t)((ed[i].info >> 2) & 3) * ne + ed[i].R] = (int32_t)((i << 1) | 1);
  }
  });
  int rc = 0;
  // the mesh in caller order (read by every regrouping) and the fixed edge data
  double *d_geo_u, *d_etb_u, *d_egeo;
  int32_t *d_eedge_u, *d_eLu, *d_eRu, *d_mem_u, *d_einfo, *d_emem;
  std::vector<float> egeo32(egeo.begin(), egeo.end());
  float* d_egeo32;
  if ((rc = upload(ctx, &d_geo_u, geo)) || (rc = upload(ctx, &d_etb_u, etb)) || (rc = upload(ctx, &d_eedge_u, eedge_u)) ||
      (rc = upload(ctx, &d_eLu, eLu)) || (rc = upload(ctx, &d_eRu, eRu)) || (rc = upload(ctx, &d_mem_u, ctx->member_user)) ||
      (rc = upload(ctx, &d_einfo, einfo)) || (rc = upload(ctx, &d_egeo, egeo)) || (rc = upload(ctx, &d_egeo32, egeo32)) ||
      (rc = upload(ctx, &d_emem, emem)))
    return cuda_err(ctx, rc);
  ctx->ms = MeshStatic{ne, nE, d_geo_u, d_etb_u, d_eedge_u, d_eLu, d_eRu, d_mem_u};
  // what the regrouping writes
  DevMeshOut& D = ctx->dout;
  if ((rc = dalloc(ctx, &D.perm, 4 * (size_t)ne)) || (rc = dalloc(ctx, &D.inv, 4 * (size_t)ne)) ||
      (rc = dalloc(ctx, &D.p, (size_t)ne)) || (rc = dalloc(ctx, &D.geo, 8 * (size_t)NGEO * ne)) ||
      (rc = dalloc(ctx, &D.geo32, 4 * (size_t)NGEO * ne)) || (rc = dalloc(ctx, &D.etb, 96 * (size_t)ne)) ||
      (rc = dalloc(ctx, &D.mem, 4 * (size_t)ne)) || (rc = dalloc(ctx, &D.eedge, 12 * (size_t)ne)) ||
      (rc = dalloc(ctx, &D.eL, 4 * (size_t)nE)) || (rc = dalloc(ctx, &D.eR, 4 * (size_t)nE)) ||
      (rc = dalloc(ctx, &D.slot, 4 * (size_t)nE)) || (rc = dalloc(ctx, &D.lists, 12 * (size_t)nE)) ||
      (rc = dalloc(ctx, &D.off, 8 * (size_t)ne)))
    return cuda_err(ctx, rc);
  {
    const int64_t be = regroup_blocks(ne), bg = regroup_blocks(nE);
    RegroupScratch& W = ctx->rw;
    if ((rc = dalloc(ctx, &W.ecnt, 4 * 5 * (size_t)be)) || (rc = dalloc(ctx, &W.eoff, 8 * 5 * (size_t)be)) ||
        (rc = dalloc(ctx, &W.gcnt, 4 * 3 * (size_t)bg)) || (rc = dalloc(ctx, &W.goff, 8 * 3 * (size_t)bg)) ||
        (rc = dalloc(ctx, &W.psum, 8 * (size_t)be)) || (rc = dalloc(ctx, &W.poff, 8 * (size_t)(be + 1))) ||
        (rc = dalloc(ctx, &W.info, 8 * 16)))
      return cuda_err(ctx, rc);
    cudaMemsetAsync(W.info, 0, 8 * 16, ctx->stream);
  }
  ctx->d_perm = D.perm;
  ctx->d_off = D.off;
  ctx->dm = DevMesh{ne, nE, nint, D.geo, D.p, D.eedge, D.eL, D.eR, d_einfo, d_egeo, D.geo32, d_egeo32, D.etb,
                    D.mem, d_emem, ctx->nmem, nullptr};
  ctx->ce.slot = D.slot;
  for (int pm = 2; pm <= 4; ++pm) ctx->ce.list[pm] = D.lists + (size_t)(pm - 2) * nE;
  // base state, velocity and fluxes (sized by the mesh)
  for (int s = 0; s < 3; ++s) {
    if ((rc = dalloc(ctx, &ctx->st[s].cb, sizeof(double) * 9 * ne))) return cuda_err(ctx, rc);
    cudaMemsetAsync(ctx->st[s].cb, 0, sizeof(double) * 9 * ne, ctx->stream);
    ctx->st[s].cb32 = nullptr;
    if (ctx->corr32) {
      if ((rc = dalloc(ctx, &ctx->st[s].cb32, sizeof(float) * 9 * ne))) return cuda_err(ctx, rc);
      cudaMemsetAsync(ctx->st[s].cb32, 0, sizeof(float) * 9 * ne, ctx->stream);
    }
  }
  if ((rc = dalloc(ctx, &ctx->vel.ub, sizeof(double) * 6 * ne))) return cuda_err(ctx, rc);
  ctx->vel.ub32 = nullptr;
  if (ctx->corr32 && (rc = dalloc(ctx, &ctx->vel.ub32, sizeof(float) * 6 * ne))) return cuda_err(ctx, rc);
  if ((rc = dalloc(ctx, &ctx->fx.Fb, sizeof(double) * 6 * nE)) || (rc = dalloc(ctx, &ctx->fx.Fbc, sizeof(double) * 6 * nE)))
    return cuda_err(ctx, rc);
  if ((rc = dalloc(ctx, &ctx->d_user, sizeof(double) * 3 * KMAX * ne)) ||
      (rc = dalloc(ctx, &ctx->d_user2, sizeof(double) * 3 * KMAX * ne)))
    return cuda_err(ctx, rc);
  if ((rc = dalloc(ctx, &ctx->d_newp, (size_t)ne))) return cuda_err(ctx, rc);
  const size_t nm = (size_t)ctx->nmem;
  if ((rc = dalloc(ctx, &ctx->d_dt, sizeof(double) * nm)) || (rc = dalloc(ctx, &ctx->d_t, sizeof(double) * nm)) ||
      (rc = dalloc(ctx, &ctx->d_dmin, sizeof(unsigned long long) * nm)) ||
      (rc = dalloc(ctx, &ctx->d_status, sizeof(unsigned))) ||
      (rc = dalloc(ctx, &ctx->d_mstatus, sizeof(unsigned) * nm)))
    return cuda_err(ctx, rc);
  cudaMemsetAsync(ctx->d_mstatus, 0, sizeof(unsigned) * nm, ctx->stream);
  cudaMemsetAsync(ctx->d_dt, 0, sizeof(double) * nm, ctx->stream);
  if ((rc = launch_reset_min(ctx->stream, ctx->d_dmin, ctx->nmem))) return cuda_err(ctx, rc);
  ctx->nred = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (ne + 255) / 256));
  if ((rc = dalloc(ctx, &ctx->d_partial, sizeof(double) * ctx->nred)) || (rc = dalloc(ctx, &ctx->d_red, sizeof(double) * 2)))
    return cuda_err(ctx, rc);
  cudaMemsetAsync(ctx->d_t, 0, sizeof(double) * nm, ctx->stream);
  cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream);
  ctx->dm.mstatus = ctx->d_mstatus;
  if ((rc = dalloc(ctx, &ctx->d_work, sizeof(unsigned) * 4))) return cuda_err(ctx, rc);
  cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned) * 4, ctx->stream);
  // the order-dependent part
  CU(cudaMemcpyAsync(ctx->d_newp, ctx->p_user.data(), (size_t)ne, cudaMemcpyHostToDevice, ctx->stream));
  ctx->packed_n = -1;
  CK(regroup(ctx, false));
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, cuda_fail(e, "build_device", __FILE__, __LINE__));
  return 0;
}

// ------------------------------------------------------------------ stages
static Phys phys(const swe_ctx* ctx) {
  const swe_params& p = ctx->prm;
  return Phys{p.g, p.h_min, p.tide_amp, p.tide_period, p.tide_phase, p.fric_lin, p.fric_quad, p.f_c,
              (p.fric_lin != 0.0 || p.fric_quad != 0.0 || p.f_c != 0.0) ? 1 : 0};
}

// The FP32 copies of the base state and velocity serve the correction kernels
// only: with no element of order >= 2 they are not written (an order change
// rewrites them from the caller layout before a correction kernel reads them).
static float* cb32_out(const swe_ctx* ctx, const StateDev& s) { return ctx->G.start[2] < ctx->ne ? s.cb32 : nullptr; }
static float* ub32_out(const swe_ctx* ctx) { return ctx->G.start[2] < ctx->ne ? ctx->vel.ub32 : nullptr; }

static int usolve_all(swe_ctx* ctx, StateDev in) {
  ProfScope ps(ctx, F_USOLVE);
  const Phys ph = phys(ctx);
  CK(launch_usolve_base(ctx->stream, ctx->dm, ctx->G, ph, in.cb, ctx->vel.ub, ub32_out(ctx), ctx->d_status, nullptr));
  if (ctx->tc)
    CK(corrtc::launch_usolve_corr(GroupStreams{{ctx->stream, ctx->stream, ctx->stream}}, ctx->dm, ctx->G, ph, in, ctx->vel,
                                  ctx->d_status, nullptr, nullptr));
  else if (ctx->corr32)
    CK(corr32::launch_usolve_corr(GroupStreams{{ctx->stream, ctx->stream, ctx->stream}}, ctx->dm, ctx->G, ph, in, ctx->vel,
                                  ctx->d_status, nullptr, nullptr));
  else CK(corr64::launch_usolve_corr(GroupStreams{{ctx->stream, ctx->stream, ctx->stream}}, ctx->dm, ctx->G, ph, in, ctx->vel,
                                  ctx->d_status, nullptr, nullptr));
  return 0;
}

// One stage: out = a n + b (in + dt L(in)), or out = L(in) (rhs_only).
//
// The base kernels (FP64 pipe bound) run on stream A, the correction kernels
// on stream B, concurrently on the same SMs -- the GB300 counterpart of the
// paper's base/correction distribution over CPU and GPU (Sect. 3-5):
//   A: usolve_base --------> [dt] edge_base -------------------------> elem_base
//   B: usolve_corr (+ rc) -->      edge_corr -> elem_corr(q >= 3) ---^
// (each edge kernel needs both u-solves; elem_base needs the rc of the base
// test modes, which the velocity solve forms, and edge_corr's share of the
// base-mode flux).  With the split schedule (a launch-shape choice) the
// higher test modes, which write only the correction part of the state, run
// beside elem_base instead:
//   B: usolve_corr (+ rc) -->      edge_corr ----> elem_corr(q >= 3) --> (join)
//   A:                        ... edge_base --^--> elem_base ------------^
// The tensor-core mode runs edge_corr -> vol_tc -> elem_corr(every q) on B
// before the join.  Profiling runs everything on A.
static int run_stage(swe_ctx* ctx, StateDev in, StateDev nst, StateDev out, const Stage& stg, bool cfl_dt,
                     double dt_fixed) {
  const Phys ph = phys(ctx);
  const bool conc = !ctx->prof;
  const bool split = ctx->shape.split && !ctx->tc && !stg.base_only;
  cudaStream_t A = ctx->stream, B = conc ? ctx->stream2 : ctx->stream;
  // the order groups of each correction launch run concurrently: forked from
  // B onto the group streams and joined back before B's next launch
  const GroupStreams gs = conc ? GroupStreams{{B, ctx->sg[0], ctx->sg[1]}} : GroupStreams{{A, A, A}};
  auto fork_groups = [&]() -> int {
    if (!conc) return 0;
    CU(cudaEventRecord(ctx->ev_gf, B));
    CU(cudaStreamWaitEvent(ctx->sg[0], ctx->ev_gf, 0));
    CU(cudaStreamWaitEvent(ctx->sg[1], ctx->ev_gf, 0));
    return 0;
  };
  auto join_groups = [&]() -> int {
    if (!conc) return 0;
    for (int i = 0; i < 2; ++i) {
      CU(cudaEventRecord(ctx->ev_gj[i], ctx->sg[i]));
      CU(cudaStreamWaitEvent(B, ctx->ev_gj[i], 0));
    }
    return 0;
  };
  if (conc) {
    CU(cudaEventRecord(ctx->ev_fork, A));
    CU(cudaStreamWaitEvent(B, ctx->ev_fork, 0));
  }
  {
    // the first stage of a CFL step folds the elements' CFL bounds into d_dmin
    ProfScope ps(ctx, F_USOLVE);
    unsigned long long* dmin = cfl_dt ? ctx->d_dmin : nullptr;
    CK(launch_usolve_base(A, ctx->dm, ctx->G, ph, in.cb, ctx->vel.ub, ub32_out(ctx), ctx->d_status, dmin));
    CK(fork_groups());
    // the CUDA-core modes form rc in the velocity solve; the tensor-core mode in elem_corr (from vol)
    if (ctx->tc) CK(corrtc::launch_usolve_corr(gs, ctx->dm, ctx->G, ph, in, ctx->vel, ctx->d_status, dmin, nullptr));
    else if (ctx->corr32)
      CK(corr32::launch_usolve_corr(gs, ctx->dm, ctx->G, ph, in, ctx->vel, ctx->d_status, dmin, ctx->rc));
    else CK(corr64::launch_usolve_corr(gs, ctx->dm, ctx->G, ph, in, ctx->vel, ctx->d_status, dmin, ctx->rc));
    CK(join_groups());
  }
  if (conc) {
    CU(cudaEventRecord(ctx->ev_u1, A));
    CU(cudaEventRecord(ctx->ev_u2, B));
    CU(cudaStreamWaitEvent(A, ctx->ev_u2, 0));
    CU(cudaStreamWaitEvent(B, ctx->ev_u1, 0));
  }
  if (cfl_dt) {
    ProfScope ps(ctx, F_DT);  // dt = cfl * min, and the minimum reset for the next step
    CK(launch_advance_time(A, nullptr, ctx->d_dmin, ctx->prm.cfl, dt_fixed, ctx->d_dt, ctx->nmem));
    if (conc) {  // the correction branch reads dt (stage time, RK update)
      CU(cudaEventRecord(ctx->ev_dt, A));
      CU(cudaStreamWaitEvent(B, ctx->ev_dt, 0));
    }
  }
  {
    ProfScope ps(ctx, F_EDGEB);
    CK(launch_edge_base(A, ctx->dm, ph, stg, in.cb, ctx->vel.ub, ctx->fx, ctx->d_work));
  }
  auto elem_corr = [&](int part) -> int {
    ProfScope ps(ctx, F_ELEMC);
    CK(fork_groups());
    if (ctx->tc)
      CK(corrtc::launch_elem_corr(gs, ctx->dm, ctx->ce, ctx->G, ph, stg, in, nst, out, ctx->vel, ctx->fx, ctx->rc,
                                  part, ctx->vol));
    else if (ctx->corr32)
      CK(corr32::launch_elem_corr(gs, ctx->dm, ctx->ce, ctx->G, ph, stg, in, nst, out, ctx->vel, ctx->fx, ctx->rc,
                                  part));
    else
      CK(corr64::launch_elem_corr(gs, ctx->dm, ctx->ce, ctx->G, ph, stg, in, nst, out, ctx->vel, ctx->fx, ctx->rc,
                                  part));
    CK(join_groups());
    return 0;
  };
  if (!stg.base_only) {
    {
      ProfScope ps(ctx, F_EDGEC);
      CK(fork_groups());
      if (ctx->tc) CK(corrtc::launch_edge_corr(gs, ctx->dm, ctx->ce, ctx->G, ph, stg, in, ctx->vel, ctx->fx));
      else if (ctx->corr32) CK(corr32::launch_edge_corr(gs, ctx->dm, ctx->ce, ctx->G, ph, stg, in, ctx->vel, ctx->fx));
      else CK(corr64::launch_edge_corr(gs, ctx->dm, ctx->ce, ctx->G, ph, stg, in, ctx->vel, ctx->fx));
      CK(join_groups());
    }
    if (ctx->tc) {  // every test mode (rc comes from the tensor-core volume terms)
      {
        ProfScope ps(ctx, F_VOLTC);
        CK(corrtc::launch_vol_tc(B, ctx->dm, ctx->G, ph, in, ctx->vel, ctx->vol, ctx->d_status));
      }
      CK(elem_corr(0));
    } else if (!split) {
      CK(elem_corr(1));  // the higher test modes (the velocity solve formed rc)
    }
  }
  if (conc) {
    CU(cudaEventRecord(ctx->ev_c, B));
    CU(cudaStreamWaitEvent(A, ctx->ev_c, 0));
  }
  if (split) CK(elem_corr(1));  // the higher test modes, beside elem_base
  {
    ProfScope ps(ctx, F_ELEMB);
    CK(launch_elem_base(A, ctx->dm, ctx->G, ph, stg, in.cb, nst.cb, out.cb, cb32_out(ctx, out), ctx->vel.ub, ctx->fx,
                        ctx->rc, ctx->d_work + 2));
  }
  if (conc && split) {
    CU(cudaEventRecord(ctx->ev_c2, B));
    CU(cudaStreamWaitEvent(A, ctx->ev_c2, 0));
  }
  return 0;
}

// One SSP-RK step of state A (in place); the step size lives in d_dt.
static int enqueue_step(swe_ctx* ctx, double dt_fixed) {
  StateDev A = ctx->st[0], B = ctx->st[1], C = ctx->st[2];
  Stage s{};
  s.dt = ctx->d_dt;
  s.t_dev = ctx->d_t;
  if (dt_fixed > 0.0) {
    ProfScope ps(ctx, F_DT);
    CK(launch_advance_time(ctx->stream, nullptr, ctx->d_dmin, ctx->prm.cfl, dt_fixed, ctx->d_dt, ctx->nmem));
  }
  const bool cfl = dt_fixed <= 0.0;
  if (ctx->prm.rk_order == 3) {
    s.a = 0.0; s.b = 1.0; s.tau = 0.0;
    CK(run_stage(ctx, A, A, B, s, cfl, dt_fixed));
    s.a = 0.75; s.b = 0.25; s.tau = 1.0;
    CK(run_stage(ctx, B, A, C, s, false, dt_fixed));
    s.a = 1.0 / 3.0; s.b = 2.0 / 3.0; s.tau = 0.5;
    CK(run_stage(ctx, C, A, A, s, false, dt_fixed));
  } else {
    s.a = 0.0; s.b = 1.0; s.tau = 0.0;
    CK(run_stage(ctx, A, A, B, s, cfl, dt_fixed));
    s.a = 0.5; s.b = 0.5; s.tau = 1.0;
    CK(run_stage(ctx, B, A, A, s, false, dt_fixed));
  }
  ProfScope ps(ctx, F_OTHER);
  CK(launch_advance_time(ctx->stream, ctx->d_t, nullptr, 0.0, 0.0, ctx->d_dt, ctx->nmem));
  return 0;
}

static int read_status(swe_ctx* ctx, bool check_state) {
  if (check_state) CK(launch_check_state(ctx->stream, ctx->dm, ctx->G, ctx->corr32, ctx->st[0], ctx->d_status));
  unsigned st = 0;
  CU(cudaMemcpyAsync(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (st) CU(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
  if (st & ST_TIMEOUT) return fail(ctx, SWE_ETIMEOUT, "a tensor-core wait ran out");
  if (st & ST_NONFINITE) return fail(ctx, SWE_ENONFINITE, "non-finite value in the state");
  if (st & ST_DEPTH) return fail(ctx, SWE_EDEPTH, "an element mean depth fell to or below h_min");
  return 0;
}

// caller layout (host or device) -> state A (or the scratch state s)
static int state_in(swe_ctx* ctx, const double* c, int s, bool packed = false) {
  const size_t bytes = sizeof(double) * (packed ? (size_t)ctx->packed_n : (size_t)3 * KMAX * ctx->ne);
  const double* src = c;
  if (!is_device_ptr(c)) {
    CU(cudaMemcpyAsync(ctx->d_user, c, bytes, cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->d_user;
  }
  CK(launch_from_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, packed ? ctx->d_off : nullptr, ctx->corr32, src,
                      ctx->st[s]));
  if (s == 0)  // a new state: the members' status starts afresh
    CU(cudaMemsetAsync(ctx->d_mstatus, 0, sizeof(unsigned) * (size_t)ctx->nmem, ctx->stream));
  return 0;
}

static int state_out(swe_ctx* ctx, StateDev st, double* c, bool packed = false) {
  const size_t bytes = sizeof(double) * (packed ? (size_t)ctx->packed_n : (size_t)3 * KMAX * ctx->ne);
  const bool dev = is_device_ptr(c);
  double* dst = dev ? c : ctx->d_user2;
  CK(launch_to_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, packed ? ctx->d_off : nullptr, ctx->corr32, st,
                    dst));
  if (!dev) CU(cudaMemcpyAsync(c, dst, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

// ------------------------------------------------------------------ ABI
extern "C" {

void swe_default_params(swe_params* p) {
  std::memset(p, 0, sizeof *p);
  p->g = 9.81;
  p->cfl = 0.1;
  p->h_min = 1e-8;
  p->rk_order = 2;
  p->precision = SWE_PREC_FP64;
}

int swe_create(swe_ctx** out, const swe_params* params) {
  if (!out || !params) { g_create_err = "swe_create: NULL argument"; return SWE_EINVAL; }
  *out = nullptr;
  if (params->rk_order != 2 && params->rk_order != 3) { g_create_err = "rk_order must be 2 or 3"; return SWE_EINVAL; }
  if (params->precision != SWE_PREC_FP64 && params->precision != SWE_PREC_MIXED_FP32 &&
      params->precision != SWE_PREC_MIXED_TF32) {
    g_create_err = "unknown precision mode"; return SWE_EINVAL;
  }
  if (!(params->g > 0.0) || !(params->cfl > 0.0)) { g_create_err = "g and cfl must be positive"; return SWE_EINVAL; }
  if (!(params->fric_lin >= 0.0) || !(params->fric_quad >= 0.0) || !std::isfinite(params->f_c)) {
    g_create_err = "friction coefficients must be >= 0 and f_c finite"; return SWE_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_create_err_s = std::string("no CUDA device: ") + cudaGetErrorString(e);
    g_create_err = g_create_err_s.c_str();
    return SWE_ECUDA;
  }
  swe_ctx* ctx = new swe_ctx;
  ctx->prm = *params;
  ctx->device = dev;
  ctx->corr32 = params->precision == SWE_PREC_MIXED_FP32 || params->precision == SWE_PREC_MIXED_TF32;
  ctx->tc = params->precision == SWE_PREC_MIXED_TF32;
  if (params->cuda_stream) {
    ctx->stream = (cudaStream_t)params->cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete ctx; g_create_err = "cudaStreamCreate failed"; return SWE_ECUDA; }
    ctx->own_stream = true;
  }
  {
    // the correction branch is the longer one: give its blocks precedence
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    e = cudaStreamCreateWithPriority(&ctx->stream2, cudaStreamNonBlocking, hi);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithPriority(&ctx->sg[i], cudaStreamNonBlocking, hi);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_u1, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_u2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_c, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_dt, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_c2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_gf, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ctx->ev_gj[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    g_create_err = "stream/event creation failed";
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return SWE_ECUDA;
  }
  {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    set_sm_count(nsm);
  }
  // the reference tables go to the device's constant memory once per process
  // (a later write would race with the kernels of contexts already running)
  {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) {
      g_create_err = "device ordinal out of range";
      e = cudaErrorInvalidDevice;
    } else if (!done[dev]) {
      upload_base_tables();
      corr64::upload_tables();
      corr32::upload_tables();
      corrtc::upload_tables();
      if (corrtc::upload_tc_tables() != 0) {
        g_create_err = "tensor-core operand upload failed";
        e = cudaErrorUnknown;
      } else {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
          g_create_err_s = std::string("table upload failed: ") + cudaGetErrorString(e);
          g_create_err = g_create_err_s.c_str();
        } else {
          done[dev] = true;
        }
      }
    }
  }
  if (e != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return SWE_ECUDA;
  }
  *out = ctx;
  return 0;
}

void swe_destroy(swe_ctx* ctx) {
  if (!ctx) return;
  sync_streams(ctx);
  free_all(ctx);
  cudaStreamSynchronize(ctx->stream);  // the frees are done before the stream goes
  for (auto& ev : ctx->evs) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
  for (auto ev : ctx->pool) cudaEventDestroy(ev);
  for (cudaEvent_t ev : {ctx->ev_fork, ctx->ev_u1, ctx->ev_u2, ctx->ev_c, ctx->ev_dt, ctx->ev_c2, ctx->ev_gf,
                         ctx->ev_gj[0], ctx->ev_gj[1]})
    if (ev) cudaEventDestroy(ev);
  if (ctx->stream2) { cudaStreamSynchronize(ctx->stream2); cudaStreamDestroy(ctx->stream2); }
  for (cudaStream_t cs : {ctx->cin, ctx->cout})
    if (cs) { cudaStreamSynchronize(cs); cudaStreamDestroy(cs); }
  for (int k = 0; k < 2; ++k)
    for (cudaEvent_t ev : {ctx->ev_in[k], ctx->ev_conv[k], ctx->ev_oready[k], ctx->ev_d2h[k]})
      if (ev) cudaEventDestroy(ev);
  for (cudaStream_t sgi : ctx->sg)
    if (sgi) { cudaStreamSynchronize(sgi); cudaStreamDestroy(sgi); }
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* swe_last_error(const swe_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err; }

int swe_set_mesh(swe_ctx* ctx, int64_t nv, const double* xy, int64_t ne, const int32_t* tri, const int8_t* bc_tag) {
  if (!ctx) return SWE_EINVAL;
  if (nv < 3 || ne < 1 || !xy || !tri) return fail(ctx, SWE_EINVAL, "swe_set_mesh: need nv >= 3, ne >= 1 and arrays");
  ctx->nv = nv; ctx->ne = ne;
  ctx->xy.assign(xy, xy + 2 * nv);
  ctx->hv.assign(nv, 0.0);
  ctx->tri.resize(3 * ne);
  ctx->tag.assign(3 * ne, 0);
  // per chunk the first bad triangle (1: vertex id, 2: boundary tag, 3: degenerate); the lowest is reported
  std::vector<std::pair<int64_t, int>> bad;
  std::mutex mu;
  host_parallel(ne, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int32_t v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
      int8_t t[3] = {0, 0, 0};
      if (bc_tag) for (int k = 0; k < 3; ++k) t[k] = bc_tag[3 * e + k];
      int why = 0;
      for (int k = 0; k < 3; ++k)
        if (v[k] < 0 || v[k] >= nv) why = 1;
      for (int k = 0; k < 3 && !why; ++k)
        if (t[k] < 0 || t[k] > 2) why = 2;
      double cr = 0.0;
      if (!why) {
        cr = (xy[2 * v[1]] - xy[2 * v[0]]) * (xy[2 * v[2] + 1] - xy[2 * v[0] + 1]) -
             (xy[2 * v[2]] - xy[2 * v[0]]) * (xy[2 * v[1] + 1] - xy[2 * v[0] + 1]);
        if (!(cr != 0.0) || !std::isfinite(cr)) why = 3;
      }
      if (why) {
        std::lock_guard<std::mutex> g(mu);
        bad.push_back({e, why});
        return;
      }
      if (cr < 0.0) { std::swap(v[1], v[2]); std::swap(t[1], t[2]); }
      for (int k = 0; k < 3; ++k) { ctx->tri[3 * e + k] = v[k]; ctx->tag[3 * e + k] = t[k]; }
    }
  });
  if (!bad.empty()) {
    const auto b = *std::min_element(bad.begin(), bad.end());
    ctx->have_mesh = false;
    if (b.second == 1) return fail(ctx, SWE_EMESH, "triangle %lld: vertex id out of range", (long long)b.first);
    if (b.second == 2) return fail(ctx, SWE_EINVAL, "triangle %lld: boundary tag must be 0, 1 or 2", (long long)b.first);
    return fail(ctx, SWE_EMESH, "triangle %lld is degenerate", (long long)b.first);
  }
  ctx->p_user.assign(ne, 1);
  ctx->member_user.assign(ne, 0);
  ctx->nmem = 1;
  int rc = build_topology(ctx);
  if (rc) { ctx->have_mesh = false; return rc; }
  ctx->have_mesh = true;
  ctx->dirty = true;
  ctx->keep_valid = false;
  std::vector<double>().swap(ctx->keep_c);
  return 0;
}

int swe_mesh_adjacency(int64_t nv, const double* xy, int64_t ne, const int32_t* tri, int32_t* nbr_out,
                       int8_t* nbk_out) {
  if (!nbr_out || ne > (int64_t)INT32_MAX) {
    g_create_err = "swe_mesh_adjacency: NULL nbr_out or ne >= 2^31";
    return SWE_EINVAL;
  }
  swe_ctx tmp;  // the host description only: swe_set_mesh touches no device
  const int rc = swe_set_mesh(&tmp, nv, xy, ne, tri, nullptr);
  if (rc) {
    g_create_err_s = tmp.err;
    g_create_err = g_create_err_s.c_str();
    return rc;
  }
  // swe_set_mesh re-orients a clockwise triangle by swapping its vertices 1
  // and 2, which swaps its local edges 1 and 2 (a swap is its own inverse)
  auto local = [&](int64_t e, int k) { return tmp.tri[3 * e + 1] != tri[3 * e + 1] && k ? 3 - k : k; };
  for (int64_t e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) {
      const int ki = local(e, k);
      const int64_t n = tmp.nb[3 * e + ki];
      nbr_out[3 * e + k] = (int32_t)n;
      if (nbk_out) nbk_out[3 * e + k] = n < 0 ? (int8_t)-1 : (int8_t)local(n, tmp.nbk[3 * e + ki]);
    }
  return 0;
}

// The device data follow the host description lazily: a setter marks the
// context dirty, keeping the current state in the caller layout when the
// device holds one, and the first call that needs the device builds it once
// (so mesh + bathymetry + orders + members cost one build).
static int mark_dirty_keep_state(swe_ctx* ctx) {
  if (!ctx->dirty) {
    ctx->keep_c.resize((size_t)3 * KMAX * ctx->ne);
    int rc = swe_get_state(ctx, ctx->keep_c.data(), &ctx->keep_t);
    if (rc) return rc;
    ctx->keep_valid = true;
  }
  ctx->dirty = true;
  return 0;
}

static int ensure_built(swe_ctx* ctx) {
  if (!ctx->dirty) return 0;
  int rc = build_device(ctx);
  if (rc) return rc;
  ctx->dirty = false;
  if (ctx->keep_valid) {
    ctx->keep_valid = false;
    rc = swe_set_state(ctx, ctx->keep_c.data(), ctx->keep_t);
    std::vector<double>().swap(ctx->keep_c);
  }
  return rc;
}

int swe_set_bathymetry(swe_ctx* ctx, const double* hb_vertex) {
  if (!ctx || !ctx->have_mesh || !hb_vertex) return fail(ctx, SWE_EINVAL, "swe_set_bathymetry: no mesh or NULL");
  for (int64_t v = 0; v < ctx->nv; ++v)
    if (!std::isfinite(hb_vertex[v])) return fail(ctx, SWE_EINVAL, "bathymetry at vertex %lld is not finite", (long long)v);
  int rc = mark_dirty_keep_state(ctx);
  if (rc) return rc;
  ctx->hv.assign(hb_vertex, hb_vertex + ctx->nv);
  return 0;
}

int swe_set_orders(swe_ctx* ctx, const int8_t* p) {
  if (!ctx || !ctx->have_mesh || !p) return fail(ctx, SWE_EINVAL, "swe_set_orders: no mesh or NULL");
  for (int64_t e = 0; e < ctx->ne; ++e)
    if (p[e] < 0 || p[e] > 4) return fail(ctx, SWE_EINVAL, "order of element %lld is %d, not in 0..4", (long long)e, (int)p[e]);
  ctx->p_user.assign(p, p + ctx->ne);
  if (ctx->dirty) return 0;  // the next build groups the elements
  // a built context regroups on the device and carries the state over
  LaunchScope ls(ctx);
  CU(cudaMemcpyAsync(ctx->d_newp, p, (size_t)ctx->ne, cudaMemcpyHostToDevice, ctx->stream));
  return regroup(ctx, true);
}

int swe_set_state(swe_ctx* ctx, const double* c, double t) {
  if (!ctx || !ctx->have_mesh || !c) return fail(ctx, SWE_EINVAL, "swe_set_state: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(state_in(ctx, c, 0));
  const std::vector<double> tv((size_t)ctx->nmem, t);
  CU(cudaMemcpyAsync(ctx->d_t, tv.data(), sizeof(double) * tv.size(), cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_get_state(swe_ctx* ctx, double* c_out, double* t_out) {
  if (!ctx || !ctx->have_mesh || !c_out) return fail(ctx, SWE_EINVAL, "swe_get_state: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(state_out(ctx, ctx->st[0], c_out));
  if (t_out) {
    CU(cudaMemcpyAsync(t_out, ctx->d_t, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  return 0;
}

int64_t swe_packed_size(swe_ctx* ctx) {
  if (!ctx || !ctx->have_mesh) return fail(ctx, SWE_EINVAL, "swe_packed_size: no mesh");
  CK(ensure_built(ctx));
  return ctx->packed_n;
}

int swe_set_state_packed(swe_ctx* ctx, const double* c, double t) {
  if (!ctx || !ctx->have_mesh || !c) return fail(ctx, SWE_EINVAL, "swe_set_state_packed: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(state_in(ctx, c, 0, true));
  const std::vector<double> tv((size_t)ctx->nmem, t);
  CU(cudaMemcpyAsync(ctx->d_t, tv.data(), sizeof(double) * tv.size(), cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_get_state_packed(swe_ctx* ctx, double* c_out, double* t_out) {
  if (!ctx || !ctx->have_mesh || !c_out) return fail(ctx, SWE_EINVAL, "swe_get_state_packed: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(state_out(ctx, ctx->st[0], c_out, true));
  if (t_out) {
    CU(cudaMemcpyAsync(t_out, ctx->d_t, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  return 0;
}

int swe_p1_modes(swe_ctx* ctx, const double* vals, double* modes_out) {
  if (!ctx || !ctx->have_mesh || !vals || !modes_out) return fail(ctx, SWE_EINVAL, "swe_p1_modes: no mesh or NULL");
  const RefTables& R = tables();
  const int64_t ne = ctx->ne;
  std::vector<double> out((size_t)3 * ne);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* v = &ctx->tri[3 * e];
    const double x0 = ctx->xy[2 * v[0]], y0 = ctx->xy[2 * v[0] + 1];
    const double det = (ctx->xy[2 * v[1]] - x0) * (ctx->xy[2 * v[2] + 1] - y0) -
                       (ctx->xy[2 * v[2]] - x0) * (ctx->xy[2 * v[1] + 1] - y0);
    const double s = std::sqrt(det);
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
      for (int w = 0; w < 3; ++w) acc += vals[v[w]] * R.Lv[w][i];
      out[(size_t)i * ne + e] = s * acc;
    }
  }
  if (is_device_ptr(modes_out)) {
    CU(cudaMemcpy(modes_out, out.data(), sizeof(double) * out.size(), cudaMemcpyHostToDevice));
  } else {
    std::memcpy(modes_out, out.data(), sizeof(double) * out.size());
  }
  return 0;
}

static int rhs_impl(swe_ctx* ctx, const double* c_in, double* out0, double* out1) {
  if (!ctx || !ctx->have_mesh || !c_in || !out0) return fail(ctx, SWE_EINVAL, "swe_rhs: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(state_in(ctx, c_in, 1));
  Stage s{};
  s.rhs_only = 1;
  s.dt = nullptr; s.dt_host = 0.0;
  s.t_dev = ctx->d_t; s.tau = 0.0;
  CK(run_stage(ctx, ctx->st[1], ctx->st[1], ctx->st[2], s, false, 0.0));
  int rc = read_status(ctx, false);
  if (rc) return rc;
  if (!out1) return state_out(ctx, ctx->st[2], out0);
  // order separation: the whole rhs, then the base part alone; corr = whole - base
  const int64_t n = 3 * KMAX * ctx->ne;
  CK(launch_to_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, nullptr, ctx->corr32, ctx->st[2], ctx->d_user));
  s.base_only = 1;
  CK(run_stage(ctx, ctx->st[1], ctx->st[1], ctx->st[2], s, false, 0.0));
  for (int p = 2; p < 5; ++p)  // the base part has no higher modes
    if (ctx->st[2].ch[p]) {
      const int64_t np = ctx->G.start[p + 1] - ctx->G.start[p];
      CU(cudaMemsetAsync(ctx->st[2].ch[p], 0, (ctx->corr32 ? 4 : 8) * 3 * (Kof(p) - 3) * np, ctx->stream));
    }
  CK(state_out(ctx, ctx->st[2], out0));
  const bool dev0 = is_device_ptr(out0), dev1 = is_device_ptr(out1);
  double* base_dev = dev0 ? out0 : ctx->d_user2;
  if (!dev0) CU(cudaMemcpyAsync(base_dev, out0, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  double* corr_dev = dev1 ? out1 : ctx->d_user2;
  CK(launch_sub(ctx->stream, ctx->d_user, base_dev, corr_dev, n));
  if (!dev1) CU(cudaMemcpyAsync(out1, corr_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_rhs(swe_ctx* ctx, const double* c_in, double* rhs_out) { return rhs_impl(ctx, c_in, rhs_out, nullptr); }

int swe_rhs_parts(swe_ctx* ctx, const double* c_in, double* base_out, double* corr_out) {
  if (!corr_out) return fail(ctx, SWE_EINVAL, "swe_rhs_parts: NULL output");
  return rhs_impl(ctx, c_in, base_out, corr_out);
}

int swe_rk_step(swe_ctx* ctx, double dt, double* dt_used) {
  if (!ctx || !ctx->have_mesh) return fail(ctx, SWE_EINVAL, "swe_rk_step: no mesh");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(enqueue_step(ctx, dt));
  if (dt_used) CU(cudaMemcpyAsync(dt_used, ctx->d_dt, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = read_status(ctx, true);
  prof_collect(ctx);
  return rc;
}

// Capture one step into a CUDA graph (replayed by swe_run); on a stream that
// cannot be captured the steps are launched directly.
static int build_graph(swe_ctx* ctx, double dt_fixed) {
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
  const int64_t before = ctx->launches;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ctx->use_graph = false;
    return 0;
  }
  const int rc = enqueue_step(ctx, dt_fixed);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->graph_launches = ctx->launches - before;
  ctx->launches = before;
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return cuda_err(ctx, cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__));
  const cudaError_t ei = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return cuda_err(ctx, cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__));
  ctx->graph_dt = dt_fixed;
  return 0;
}

// nsteps steps enqueued on the context stream (graph replays when possible)
static int enqueue_run(swe_ctx* ctx, int64_t nsteps, double dt_fixed) {
  if (ctx->use_graph && !ctx->prof && nsteps > 0) {
    if (!ctx->graph || ctx->graph_dt != dt_fixed) CK(build_graph(ctx, dt_fixed));
  }
  if (ctx->use_graph && !ctx->prof && ctx->graph) {
    for (int64_t s = 0; s < nsteps; ++s) {
      CU(cudaGraphLaunch(ctx->graph, ctx->stream));
      ctx->launches += ctx->graph_launches;
    }
  } else {
    for (int64_t s = 0; s < nsteps; ++s) CK(enqueue_step(ctx, dt_fixed));
  }
  return 0;
}

int swe_run(swe_ctx* ctx, int64_t nsteps, double dt_fixed, double* t_out) {
  if (!ctx || !ctx->have_mesh || nsteps < 0) return fail(ctx, SWE_EINVAL, "swe_run: no mesh or negative count");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(enqueue_run(ctx, nsteps, dt_fixed));
  int rc = read_status(ctx, true);
  prof_collect(ctx);
  if (t_out) {
    CU(cudaMemcpyAsync(t_out, ctx->d_t, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  return rc;
}

// ---- asynchronous packed transfers and steps ----
static int ensure_async(swe_ctx* ctx) {
  if (!ctx->cin) {
    CU(cudaStreamCreateWithFlags(&ctx->cin, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&ctx->cout, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k)
      for (cudaEvent_t* ev : {&ctx->ev_in[k], &ctx->ev_conv[k], &ctx->ev_oready[k], &ctx->ev_d2h[k]}) {
        CU(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
        CU(cudaEventRecord(*ev, ctx->stream));  // every slot starts free
      }
  }
  bool fresh = false;
  for (int k = 0; k < 2; ++k) {
    if (!ctx->d_stage_in[k]) {
      int rc = dalloc(ctx, &ctx->d_stage_in[k], sizeof(double) * (size_t)std::max<int64_t>(ctx->packed_n, 1));
      if (!rc) rc = dalloc(ctx, &ctx->d_stage_out[k], sizeof(double) * (size_t)std::max<int64_t>(ctx->packed_n, 1));
      if (rc) return cuda_err(ctx, rc);
      fresh = true;
    }
  }
  if (fresh) CU(cudaStreamSynchronize(ctx->stream));  // the copy streams use them next
  return 0;
}

int swe_set_state_packed_async(swe_ctx* ctx, const double* c, double t) {
  if (!ctx || !ctx->have_mesh || !c) return fail(ctx, SWE_EINVAL, "swe_set_state_packed_async: no mesh or NULL");
  CK(ensure_built(ctx));
  CK(ensure_async(ctx));
  LaunchScope ls(ctx);
  const double* src = c;
  if (!is_device_ptr(c)) {
    const int k = ctx->in_slot;
    ctx->in_slot ^= 1;
    // the staging buffer is free once the conversion that last read it has run
    CU(cudaStreamWaitEvent(ctx->cin, ctx->ev_conv[k], 0));
    CU(cudaMemcpyAsync(ctx->d_stage_in[k], c, sizeof(double) * (size_t)ctx->packed_n, cudaMemcpyHostToDevice,
                       ctx->cin));
    CU(cudaEventRecord(ctx->ev_in[k], ctx->cin));
    CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_in[k], 0));
    src = ctx->d_stage_in[k];
    CK(launch_from_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, ctx->d_off, ctx->corr32, src, ctx->st[0]));
    CU(cudaEventRecord(ctx->ev_conv[k], ctx->stream));
  } else {
    CK(launch_from_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, ctx->d_off, ctx->corr32, src, ctx->st[0]));
  }
  CK(launch_fill(ctx->stream, ctx->d_t, t, ctx->nmem));
  CU(cudaMemsetAsync(ctx->d_mstatus, 0, sizeof(unsigned) * (size_t)ctx->nmem, ctx->stream));
  return 0;
}

int swe_run_async(swe_ctx* ctx, int64_t nsteps, double dt_fixed) {
  if (!ctx || !ctx->have_mesh || nsteps < 0) return fail(ctx, SWE_EINVAL, "swe_run_async: no mesh or negative count");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  return enqueue_run(ctx, nsteps, dt_fixed);
}

int swe_get_state_packed_async(swe_ctx* ctx, double* c_out) {
  if (!ctx || !ctx->have_mesh || !c_out) return fail(ctx, SWE_EINVAL, "swe_get_state_packed_async: no mesh or NULL");
  CK(ensure_built(ctx));
  CK(ensure_async(ctx));
  LaunchScope ls(ctx);
  if (is_device_ptr(c_out)) {
    CK(launch_to_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, ctx->d_off, ctx->corr32, ctx->st[0], c_out));
    return 0;
  }
  const int k = ctx->out_slot;
  ctx->out_slot ^= 1;
  // the staging buffer is free once its previous copy to the host has run
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_d2h[k], 0));
  CK(launch_to_user(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, ctx->d_off, ctx->corr32, ctx->st[0],
                    ctx->d_stage_out[k]));
  CU(cudaEventRecord(ctx->ev_oready[k], ctx->stream));
  CU(cudaStreamWaitEvent(ctx->cout, ctx->ev_oready[k], 0));
  CU(cudaMemcpyAsync(c_out, ctx->d_stage_out[k], sizeof(double) * (size_t)ctx->packed_n, cudaMemcpyDeviceToHost,
                     ctx->cout));
  CU(cudaEventRecord(ctx->ev_d2h[k], ctx->cout));
  return 0;
}

int swe_sync(swe_ctx* ctx) {
  if (!ctx) return SWE_EINVAL;
  if (!ctx->have_mesh || ctx->dirty) return 0;  // nothing was enqueued on a device description
  LaunchScope ls(ctx);
  for (cudaStream_t cs : {ctx->cin, ctx->cout})
    if (cs) CU(cudaStreamSynchronize(cs));
  return read_status(ctx, true);
}

int swe_adapt(swe_ctx* ctx, double theta_up, double theta_down, int p_min, int p_max, int64_t* n_changed,
              int8_t* orders_out) {
  if (!ctx || !ctx->have_mesh) return fail(ctx, SWE_EINVAL, "swe_adapt: no mesh");
  CK(ensure_built(ctx));
  if (p_min < 0 || p_max > 4 || p_min > p_max || !(theta_down <= theta_up))
    return fail(ctx, SWE_EINVAL, "swe_adapt: need 0 <= p_min <= p_max <= 4 and theta_down <= theta_up");
  LaunchScope ls(ctx);
  CK(launch_indicator(ctx->stream, ctx->dm, ctx->G, ctx->d_perm, ctx->corr32, ctx->st[0], theta_up, theta_down,
                      p_min, p_max, ctx->d_newp));
  std::vector<int8_t> np((size_t)ctx->ne);
  CU(cudaMemcpyAsync(np.data(), ctx->d_newp, (size_t)ctx->ne, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  int64_t changed = 0;
  for (int64_t e = 0; e < ctx->ne; ++e) changed += np[e] != ctx->p_user[e];
  if (n_changed) *n_changed = changed;
  if (orders_out) std::memcpy(orders_out, np.data(), (size_t)ctx->ne);
  if (changed == 0) return 0;
  // the new orders are in d_newp already: regroup on the device
  ctx->p_user.swap(np);
  return regroup(ctx, true);
}

int swe_run_adaptive(swe_ctx* ctx, int64_t nsteps, int64_t every, double dt_fixed, double theta_up,
                     double theta_down, int p_min, int p_max, double* t_out) {
  if (!ctx || !ctx->have_mesh || nsteps < 0 || every < 1) return fail(ctx, SWE_EINVAL, "swe_run_adaptive: bad arguments");
  CK(ensure_built(ctx));
  int64_t done = 0;
  while (done < nsteps) {
    const int64_t n = std::min(every, nsteps - done);
    int rc = swe_run(ctx, n, dt_fixed, t_out);
    if (rc) return rc;
    done += n;
    if (done % every == 0 && (rc = swe_adapt(ctx, theta_up, theta_down, p_min, p_max, nullptr, nullptr))) return rc;
  }
  return 0;
}

int swe_set_members(swe_ctx* ctx, int32_t nmembers, const int32_t* member) {
  if (!ctx || !ctx->have_mesh || nmembers < 1 || (nmembers > 1 && !member))
    return fail(ctx, SWE_EINVAL, "swe_set_members: no mesh, nmembers < 1 or NULL");
  std::vector<int32_t> mv((size_t)ctx->ne, 0);
  if (member) mv.assign(member, member + ctx->ne);
  for (int64_t e = 0; e < ctx->ne; ++e)
    if (mv[e] < 0 || mv[e] >= nmembers)
      return fail(ctx, SWE_EINVAL, "member of element %lld is %d, not in 0..%d", (long long)e, mv[e], nmembers - 1);
  for (int64_t e = 0; e < ctx->ne; ++e)
    for (int k = 0; k < 3; ++k) {
      const int64_t n = ctx->nb[3 * e + k];
      if (n >= 0 && mv[n] != mv[e])
        return fail(ctx, SWE_EINVAL, "elements %lld and %lld share an edge but not a member", (long long)e, (long long)n);
    }
  int rc = mark_dirty_keep_state(ctx);
  if (rc) return rc;
  ctx->member_user = mv;
  ctx->nmem = nmembers;
  return 0;
}

int swe_set_member_times(swe_ctx* ctx, const double* t) {
  if (!ctx || !ctx->have_mesh || !t) return fail(ctx, SWE_EINVAL, "swe_set_member_times: no mesh or NULL");
  CK(ensure_built(ctx));
  CU(cudaMemcpyAsync(ctx->d_t, t, sizeof(double) * ctx->nmem, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_get_member_times(swe_ctx* ctx, double* t_out, double* dt_out) {
  if (!ctx || !ctx->have_mesh || !t_out) return fail(ctx, SWE_EINVAL, "swe_get_member_times: no mesh or NULL");
  CK(ensure_built(ctx));
  CU(cudaMemcpyAsync(t_out, ctx->d_t, sizeof(double) * ctx->nmem, cudaMemcpyDeviceToHost, ctx->stream));
  if (dt_out) CU(cudaMemcpyAsync(dt_out, ctx->d_dt, sizeof(double) * ctx->nmem, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_member_status(swe_ctx* ctx, uint32_t* status_out) {
  if (!ctx || !ctx->have_mesh || !status_out) return fail(ctx, SWE_EINVAL, "swe_member_status: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  // set by the steps' depth checks and by the state check of swe_run / swe_rk_step / swe_sync
  CU(cudaMemcpyAsync(status_out, ctx->d_mstatus, sizeof(unsigned) * (size_t)ctx->nmem, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CU(cudaMemsetAsync(ctx->d_mstatus, 0, sizeof(unsigned) * (size_t)ctx->nmem, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_memory_bytes(swe_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return SWE_EINVAL;
  if (ctx->have_mesh) CK(ensure_built(ctx));
  *bytes = ctx->dev_bytes;
  return 0;
}

int swe_mass(swe_ctx* ctx, double* m) {
  if (!ctx || !ctx->have_mesh || !m) return fail(ctx, SWE_EINVAL, "swe_mass: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(launch_mass(ctx->stream, ctx->dm, ctx->st[0].cb, ctx->d_partial, ctx->nred, ctx->d_red));
  CU(cudaMemcpyAsync(m, ctx->d_red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return 0;
}

int swe_energy(swe_ctx* ctx, double* en) {
  if (!ctx || !ctx->have_mesh || !en) return fail(ctx, SWE_EINVAL, "swe_energy: no mesh or NULL");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(usolve_all(ctx, ctx->st[0]));
  CK(launch_energy(ctx->stream, ctx->dm, ctx->G, ctx->corr32, phys(ctx), ctx->st[0], ctx->vel, ctx->d_partial,
                   ctx->nred, ctx->d_red));
  CU(cudaMemcpyAsync(en, ctx->d_red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return read_status(ctx, false);
}

int swe_reference_tensors(double* D, double* G, double* T) {
  const RefTables& R = tables();
  if (D) std::memcpy(D, R.D, sizeof R.D);
  if (G) std::memcpy(G, R.G, sizeof R.G);
  if (T) std::memcpy(T, R.T, sizeof R.T);
  return 0;
}

int swe_edge_table(int npts, double* s, double* w, double* B) {
  if (npts < 1 || npts > 8) return SWE_EINVAL;
  const RefTables& R = tables();
  for (int g = 0; g < npts; ++g) {
    if (s) s[g] = R.es[npts][g];
    if (w) w[g] = R.ew[npts][g];
  }
  if (B)
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < KMAX; ++i)
        for (int g = 0; g < npts; ++g) B[(k * KMAX + i) * npts + g] = R.EB[npts][k][i][g];
  return 0;
}

int64_t swe_tc_operand_image(int K, float* out, int64_t cap) {
  const int64_t n = corrtc::tc_operand_image(K, out, cap);
  return n < 0 ? SWE_EINVAL : n;
}

static bool shape_ok(const int32_t* v) {
  return v[0] >= 0 && v[0] <= 32 && v[1] >= 32 && v[1] <= 128 && v[1] % 32 == 0 && v[2] >= 32 && v[2] <= 256 &&
         v[2] % 32 == 0 && v[3] >= 32 && v[3] <= 128 && v[3] % 32 == 0 && (v[4] == 0 || v[4] == 1) && v[5] >= 0 &&
         v[5] <= 16;
}

int swe_get_launch_shape(swe_ctx* ctx, int32_t* shape) {
  if (!ctx || !shape) return SWE_EINVAL;
  shape[0] = ctx->shape.base_bpsm; shape[1] = ctx->shape.base_threads;
  shape[2] = ctx->shape.usolve_threads; shape[3] = ctx->shape.corr_threads; shape[4] = ctx->shape.split;
  shape[5] = ctx->shape.base_chunk;
  return 0;
}

int swe_set_launch_shape(swe_ctx* ctx, const int32_t* shape) {
  if (!ctx || !shape || !shape_ok(shape)) return fail(ctx, SWE_EINVAL, "swe_set_launch_shape: shape out of range");
  ctx->shape = LaunchShape{shape[0], shape[1], shape[2], shape[3], shape[4], shape[5]};
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }  // captured with the old shape
  return 0;
}

// Coordinate descent over the launch shape: every candidate runs `steps` CFL
// steps from the same saved state (graph captured first, then timed with CUDA
// events on the context stream); the fastest is kept, the state and member
// times are restored.
int swe_autotune(swe_ctx* ctx, int steps, int32_t* shape_out, double* ms_out) {
  if (!ctx || !ctx->have_mesh || steps < 1) return fail(ctx, SWE_EINVAL, "swe_autotune: no mesh or steps < 1");
  CK(ensure_built(ctx));
  const size_t n = (size_t)3 * KMAX * ctx->ne;
  double* save = nullptr;
  CU(cudaMalloc(&save, sizeof(double) * n));
  std::vector<double> tm((size_t)ctx->nmem);
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = swe_get_state(ctx, save, nullptr);
  if (!rc) rc = swe_get_member_times(ctx, tm.data(), nullptr);
  if (!rc && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
    rc = fail(ctx, SWE_ECUDA, "swe_autotune: event creation failed");
  auto restore = [&]() -> int {
    int r = swe_set_state(ctx, save, 0.0);
    return r ? r : swe_set_member_times(ctx, tm.data());
  };
  auto measure = [&](const LaunchShape& sh, double* ms) -> int {
    ctx->shape = sh;
    if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
    int r = restore();
    if (!r) r = swe_run(ctx, 1, 0.0, nullptr);  // capture and warm up
    if (r) return r;
    if (cudaEventRecord(a, ctx->stream) != cudaSuccess) return fail(ctx, SWE_ECUDA, "cudaEventRecord");
    r = swe_run(ctx, steps, 0.0, nullptr);
    if (r) return r;
    if (cudaEventRecord(b, ctx->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
      return fail(ctx, SWE_ECUDA, "cudaEventSynchronize");
    float f = 0.0f;
    cudaEventElapsedTime(&f, a, b);
    *ms = f / steps;
    return 0;
  };
  LaunchShape best = ctx->shape;
  double best_ms = 0.0;
  if (!rc) rc = measure(best, &best_ms);
  const std::vector<int> cand[6] = {{1, 2, 3, 4, 6, 0}, {64, 128}, {128, 256}, {64, 128}, {0, 1}, {0, 1, 2, 4}};
  for (int k = 0; k < 6 && !rc; ++k)
    for (int v : cand[k]) {
      if (k == 4 && ctx->tc) break;   // the tensor-core mode has one schedule
      if (k == 5 && best.base_bpsm == 0) break;  // an uncapped grid has no tile schedule
      LaunchShape sh = best;
      int* f = k == 0 ? &sh.base_bpsm : k == 1 ? &sh.base_threads : k == 2 ? &sh.usolve_threads
             : k == 3 ? &sh.corr_threads : k == 4 ? &sh.split : &sh.base_chunk;
      if (*f == v) continue;
      *f = v;
      double ms = 0.0;
      if ((rc = measure(sh, &ms))) break;
      if (ms < best_ms) { best_ms = ms; best = sh; }
    }
  ctx->shape = best;
  if (ctx->graph) { cudaGraphExecDestroy(ctx->graph); ctx->graph = nullptr; }
  const int rr = restore();
  if (!rc) rc = rr;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(save);
  if (rc) return rc;
  if (shape_out) swe_get_launch_shape(ctx, shape_out);
  if (ms_out) *ms_out = best_ms;
  return 0;
}

int swe_selftest_wait(swe_ctx* ctx, int64_t spins) {
  if (!ctx || !ctx->have_mesh || spins < 1 || spins > (int64_t)1 << 20)
    return fail(ctx, SWE_EINVAL, "swe_selftest_wait: no mesh or spins out of 1..2^20");
  CK(ensure_built(ctx));
  LaunchScope ls(ctx);
  CK(corrtc::launch_wait_selftest(ctx->stream, spins, ctx->d_status));
  return read_status(ctx, false);
}

int swe_profile(swe_ctx* ctx, int enable) {
  if (!ctx) return SWE_EINVAL;
  ctx->prof = enable != 0;
  ctx->launches = 0;
  for (int f = 0; f < NFAM; ++f) { ctx->prof_ms[f] = 0.0; ctx->prof_n[f] = 0; }
  return 0;
}

int swe_profile_read(swe_ctx* ctx, int n, const char** names, double* ms, int64_t* launches) {
  if (!ctx) return SWE_EINVAL;
  prof_collect(ctx);
  int k = 0;
  for (int f = 0; f < NFAM && k < n; ++f, ++k) {
    if (names) names[k] = kFamilies[f];
    if (ms) ms[k] = ctx->prof_ms[f];
    if (launches) launches[k] = ctx->prof_n[f];
  }
  if (k < n) {  // every kernel launched since swe_profile(ctx, .)
    if (names) names[k] = "kernels";
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = ctx->launches;
    ++k;
  }
  return k;
}

}  // extern "C"
