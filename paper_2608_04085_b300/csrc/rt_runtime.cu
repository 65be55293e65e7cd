// rt_runtime.cu -- host runtime behind the C ABI of include/rt_cnop.h.
//
// Owns the device memory of a batch of RT instances (state slots, adjoint
// slots, checkpoints, dt records), drives the time loop (two stage kernels
// per step, no host synchronisation inside the loop), the checkpointed
// reverse sweep of the gradient (Sec. 3.4: exact discrete gradient with
// checkpointing), and the projected spectral-gradient CNOP loop.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rt_cnop.h"
#include "rt_internal.h"
#include "rt_launch.h"
#include "rt_revolve.h"
#include "rt_tma_plan.h"
#include "rt_spectra.h"

// The Python binding mirrors these layouts with ctypes.
static_assert(sizeof(rt_problem) == 152, "rt_problem layout");
static_assert(sizeof(rt_options) == 32, "rt_options layout");
static_assert(sizeof(rt_run_stats) == 48, "rt_run_stats layout");
static_assert(sizeof(cnop_params) == 96, "cnop_params layout");
static_assert(sizeof(cnop_result) == 64, "cnop_result layout");

using rt::InstDev;
using rt::RunDev;

// Instantiated CUDA graph of a chunk of time-step launches, keyed by
// everything that is baked into its kernel arguments.
struct GraphKey {
  int what, kind, mode, variant, lim, S, a, b;
  bool operator<(const GraphKey& o) const {
    return std::tie(what, kind, mode, variant, lim, S, a, b) <
           std::tie(o.what, o.kind, o.mode, o.variant, o.lim, o.S, o.a, o.b);
  }
};
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
  long long kind_launches[3] = {0, 0, 0};
};

// Halo copy between two slabs of one problem: 3 rows of every conserved
// plane (or cotangent plane) from the source slab's rows to the target
// slab's halo rows, in state-slot elements.
struct HaloCopy {
  long long dst_cell_off, src_cell_off;  // device instances' cell offsets
  long long dst_cells, src_cells;        // their plane sizes (held rows x nx)
  int dst_row, src_row, nx;
};
constexpr int kSlabHalo = 3;  // rows: the adjoint reads the state 3 rows out, the stages 2

struct rt_ctx {
  int n_inst = 0;                      // problems
  int n_dev = 0;                       // device instances: problems, or their y-slabs
  std::vector<int> dev_first, dev_count;  // device instances of each problem
  std::vector<HaloCopy> halos;         // halo copies between slabs (empty without slabs)
  InstDev* d_pinst = nullptr;          // per problem, tile range over all its slabs (sums over a problem)
  rt_options opt{};
  cudaStream_t stream = nullptr;       // the context's own stream (capturable)
  cudaStream_t user_stream = nullptr;  // the caller's stream; work is ordered after it
  cudaEvent_t ev_in = nullptr;
  bool graphs = true;
  std::map<GraphKey, GraphEntry> gcache;
  int device = 0;
  std::vector<rt_problem> prob;
  std::vector<InstDev> h_inst;
  InstDev* d_inst = nullptr;
  std::vector<int4> h_tiles;   // tiles of 16 rows: every tile kernel's work list
  int4* d_tiles = nullptr;
  int ntiles = 0;
  std::vector<int4> h_tiles_h[3];  // tile-stage work lists of 8, 16 (= h_tiles) and 32 rows
  int4* d_tiles_h[3] = {nullptr, nullptr, nullptr};
  int ntiles_h[3] = {0, 0, 0};
  std::vector<int4> h_tiles_a24;   // adjoint work list of 24-row tiles (FP32)
  int4* d_tiles_a24 = nullptr;
  int ntiles_a24 = 0;
  int adj_rows = 16;               // adjoint tile height in use: 16, or 24 (FP32)
  double adj_tune_ms[2] = {0, 0};  // adjoint autotuner: ms per launch with 16- and 24-row tiles
  std::vector<int4> h_strips;  // sweep-kernel strips over all instances
  int4* d_strips = nullptr;
  int nstrips = 0;
  long long total_cells = 0;
  size_t total_v = 0;
  std::vector<long long> cell_off;  // per device instance
  std::vector<long long> v_off;     // per problem
  size_t esz = 8;          // bytes per state element
  size_t slot_bytes = 0;   // one state of every instance
  double* d_base = nullptr;  // rho0 / p0 of all instances
  float* d_base_f = nullptr; // the same rounded to FP32: the base the FP32 state deviates from
  std::vector<float> h_base_f;
  long long base_rows = 0;   // rows of all instances (p0_f starts at d_base_f + base_rows)
  std::vector<long long> row_off;
  double* d_ek0 = nullptr;   // baseline e_k (anomaly objective) or null
  double* d_ek = nullptr;    // e_k scratch
  void* sA = nullptr;        // forward ping-pong
  void* sB = nullptr;
  void* sU1 = nullptr;       // stage-1 state
  void* lA = nullptr;        // adjoint ping-pong
  void* lB = nullptr;
  void* l1 = nullptr;        // stage-1 cotangent
  std::vector<void*> pool;   // checkpoint / stored-state slots
  std::vector<void*> pool1;  // stored stage-1 states (U1) of the steps the reverse sweep walks
  void** d_tab = nullptr;    // device table of slot pointers
  int tab_cap = 0;
  RunDev run{};
  double* d_partials = nullptr;  // [ntiles * 2]
  double* d_sums = nullptr;      // [n_inst * 2]
  double* d_scal = nullptr;      // [n_inst * 4] per-instance scalars for field kernels
  double* d_v = nullptr;         // perturbation (device copy)
  double* d_g = nullptr;         // gradient
  double* d_w1 = nullptr;        // CNOP work fields
  double* d_w2 = nullptr;
  double* d_w3 = nullptr;
  double* d_w4 = nullptr;
  double* d_pairs = nullptr;     // L-BFGS (s, y) ring: 2 * pairs_m fields
  double* d_blast = nullptr;     // [n_inst] step-control cotangent of the horizon-clipped last step
  double* d_coef = nullptr;      // [n_inst] coefficient of the step-control term of the current step
  int2* d_rows = nullptr;        // (instance, y) of every row of every instance (diagnostics)
  double2* d_rowsum = nullptr;   // per-row sums of rho and e_k
  double* d_sample = nullptr;    // [n_inst][4] one diagnostics sample
  int total_rows = 0;
  int pairs_m = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
  // last run
  bool have_run = false;
  int last_steps = 0;
  int last_kind = 0;         // 0: ping-pong final state; 2: stored slots
  std::vector<int> h_nstep;
  double mem_cap = 0.0;
  // launch accounting and sampled kernel timing (0: stage 1, 1: stage 2, 2: adjoint)
  long long launches = 0;
  long long kind_launches[3] = {0, 0, 0};
  int time_every = 0;
  std::vector<cudaEvent_t> evpool;
  std::vector<std::pair<int, int>> evused;  // (kind, index of the start event; end = index + 1)
  double kind_ms[3] = {0, 0, 0};
  long long kind_samples[3] = {0, 0, 0};
  int kind_pairs[3] = {0, 0, 0};  // event pairs in use per kind (each kind gets a third of the pool)
  // stage-kernel variant in use and the autotuner's timings (ms per step)
  int stage_variant = rt::STAGE_SWEEP;
  int lim = -1;  // limiter shared by every instance (compile-time specialised kernels), or -1
  // the first failure of the current call (RT_ENONFINITE / RT_ETIMEOUT), for rt_run_stats
  int bad_instance = -1, bad_step = -1;
  long long bad_cell = -1;
  double tune_ms[5] = {0, 0, 0, 0, 0};  // by variant: sweep, tile 16, tile 8, tile 32
  // TMA groups: runs of consecutive device instances of one grid shape whose
  // tiles the tile kernels fetch with tensor copies (InstDev::tma_g)
  std::vector<rt::TmaRun> tma_groups;
};

namespace {

const double kMaxFinite = 1e300;

// NVTX range over a scope (or up to end()), for tracing tools (nsys,
// ncu --nvtx); without a tool attached the calls do nothing. The ranges mark
// the host-side submission of the work, which runs asynchronously.
struct Range {
  bool open = true;
  explicit Range(const char* name) { nvtxRangePushA(name); }
  void end() {
    if (open) nvtxRangePop();
    open = false;
  }
  ~Range() { end(); }
};

rt_status fail(rt_ctx* c, rt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, RT_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                    \
  } while (0)

#define CHK(expr)                   \
  do {                              \
    rt_status s_ = (expr);          \
    if (s_ != RT_OK) return s_;     \
  } while (0)

// Sec. 2.2, Eq. rho0: tanh density at cell centres and the hydrostatic
// pressure integrated in closed form from the anchor p(y_ref) = p_ref:
// p0(y) = p_ref + g_y [ (rho_h+rho_l)/2 (y - y_ref)
//                      + (rho_h-rho_l)/2 h_s (ln cosh z - ln cosh z_ref) ],
// z = (y - y_int)/h_s, with ln cosh z = |z| + log1p(exp(-2|z|)) - ln 2.
double lncosh_no_ln2(double z) {
  const double a = std::fabs(z);
  return a + std::log1p(std::exp(-2.0 * a));
}

void base_state(const rt_problem& P, std::vector<double>& rho0, std::vector<double>& p0) {
  const double dy = (P.y1 - P.y0) / P.ny;
  const double zr = (P.y_ref - P.y_int) / P.h_s;
  rho0.resize(P.ny);
  p0.resize(P.ny);
  for (int j = 0; j < P.ny; ++j) {
    const double y = P.y0 + (j + 0.5) * dy;
    const double z = (y - P.y_int) / P.h_s;
    rho0[j] = 0.5 * (P.rho_heavy + P.rho_light) + 0.5 * (P.rho_heavy - P.rho_light) * std::tanh(z);
    const double I = 0.5 * (P.rho_heavy + P.rho_light) * (y - P.y_ref) +
                     0.5 * (P.rho_heavy - P.rho_light) * P.h_s * (lncosh_no_ln2(z) - lncosh_no_ln2(zr));
    p0[j] = P.p_ref + P.g_y * I;
  }
}

rt_status validate(rt_ctx* c, const rt_problem& P, int i) {
  if (P.nx < 4 || P.ny < 2) return fail(c, RT_EINVAL, "instance %d: need nx >= 4 and ny >= 2", i);
  if (!(P.x1 > P.x0) || !(P.y1 > P.y0)) return fail(c, RT_EINVAL, "instance %d: empty domain", i);
  if (!(P.gamma > 1.0)) return fail(c, RT_EINVAL, "instance %d: gamma must exceed 1", i);
  if (!(P.rho_heavy > 0.0) || !(P.rho_light > 0.0) || !(P.h_s > 0.0))
    return fail(c, RT_EINVAL, "instance %d: densities and h_s must be positive", i);
  if (!(P.cfl > 0.0) || P.cfl > 1.0) return fail(c, RT_EINVAL, "instance %d: cfl must be in (0, 1]", i);
  if (P.nsteps <= 0 && !(P.T > 0.0)) return fail(c, RT_EINVAL, "instance %d: need nsteps > 0 or T > 0", i);
  if (P.bc_y != RT_BC_REFLECT && P.bc_y != RT_BC_HYDROSTATIC) return fail(c, RT_EINVAL, "instance %d: bc_y", i);
  if (P.limiter < 0 || P.limiter > 2) return fail(c, RT_EINVAL, "instance %d: limiter", i);
  if (P.perturb_ncomp != 1 && P.perturb_ncomp != 2) return fail(c, RT_EINVAL, "instance %d: perturb_ncomp", i);
  if (P.flux < RT_FLUX_HLLC || P.flux > RT_FLUX_HYBRID) return fail(c, RT_EINVAL, "instance %d: flux", i);
  if (P.flux == RT_FLUX_HYBRID && !(P.flux_theta >= 1.0))
    return fail(c, RT_EINVAL, "instance %d: flux_theta must be >= 1", i);
  if (P.objective != RT_OBJ_KE && P.objective != RT_OBJ_EK_ANOMALY_L2)
    return fail(c, RT_EINVAL, "instance %d: objective", i);
  std::vector<double> r, p;
  base_state(P, r, p);
  for (int j = 0; j < P.ny; ++j)
    if (!(p[j] > 0.0)) return fail(c, RT_EINVAL, "instance %d: base pressure not positive at row %d", i, j);
  return RT_OK;
}

template <class T> T* slotp(void* p) { return static_cast<T*>(p); }

// Start/stop a sampled timing window around one time-step kernel launch.
int timing_begin(rt_ctx* c, int kind) {
  ++c->launches;
  const long long k = c->kind_launches[kind]++;
  if (c->time_every <= 0 || k % c->time_every != 0) return -1;
  const int idx = (int)(2 * c->evused.size());
  if (idx + 1 >= (int)c->evpool.size() || c->kind_pairs[kind] >= (int)(c->evpool.size() / 6)) return -1;
  ++c->kind_pairs[kind];
  cudaEventRecord(c->evpool[idx], c->stream);
  c->evused.push_back({kind, idx});
  return idx;
}
void timing_end(rt_ctx* c, int idx) {
  if (idx >= 0) cudaEventRecord(c->evpool[idx + 1], c->stream);
}

// Refresh the halo rows of every slab in `slot` (a state or cotangent slot)
// from the neighbouring slabs' rows; nothing without slabs. Plain
// device-to-device copies on the context's stream (captured into graphs).
cudaError_t exchange(rt_ctx* c, void* slot) {
  char* b = static_cast<char*>(slot);
  const size_t es = c->esz;
  for (const HaloCopy& h : c->halos) {
    const cudaError_t e = cudaMemcpy2DAsync(
        b + (4 * h.dst_cell_off + (long long)h.dst_row * h.nx) * es, (size_t)h.dst_cells * es,
        b + (4 * h.src_cell_off + (long long)h.src_row * h.nx) * es, (size_t)h.src_cells * es,
        (size_t)kSlabHalo * h.nx * es, 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------ TMA tensor maps
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver (null if the driver lacks it).
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Map of group g over a state slot at `slot`: the 4-D tensor (x, y, component,
// instance) with boxes of TMA_BOX_X x rows x 4 x 1. Host-side encoding only.
bool encode_group(const rt_ctx* c, const rt::TmaRun& g, const void* slot, int rows, CUtensorMap* m) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t es = c->esz, plane = (cuuint64_t)g.nx * g.ny * es;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 4, (cuuint64_t)g.count};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, plane, 4 * plane};
  const cuuint32_t box[4] = {(cuuint32_t)rt::TMA_BOX_X, (cuuint32_t)rows, 4, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  void* base = const_cast<char*>(static_cast<const char*>(slot)) + 4 * c->cell_off[g.first] * (long long)es;
  return enc(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of every TMA group over `slot` with boxes of `rows` rows (all zero, and
// never read, without groups).
cudaError_t tile_maps(const rt_ctx* c, const void* slot, int rows, rt::TileMaps& m) {
  std::memset(&m, 0, sizeof(m));
  for (size_t g = 0; g < c->tma_groups.size(); ++g)
    if (!encode_group(c, c->tma_groups[g], slot, rows, &m.m[g])) return cudaErrorInvalidValue;
  return cudaSuccess;
}

// Box rows of the tile stage kernels (tile height + 2 ghost rows each side)
// and of the adjoint's state (3) and cotangent (2) tiles, for adjoint tiles
// of 16 and 24 rows.
constexpr int kStageBoxRows[3] = {8 + 4, rt::TILE_Y + 4, 32 + 4};
constexpr int kAdjBoxRowsU[2] = {16 + 6, 24 + 6}, kAdjBoxRowsK[2] = {16 + 4, 24 + 4};

// Smallest grid that holds a box of every kind: TMA_BOX_X + TILE_X columns,
// the rows of the tallest box.
constexpr int kTmaMinNx = rt::TMA_BOX_X + rt::TILE_X, kTmaMinNy = kStageBoxRows[2];

// TMA groups of the device instances (rt_tma_plan.h), kept when their maps
// encode.
void assign_tma_groups(rt_ctx* c) {
  c->tma_groups.clear();
  for (InstDev& I : c->h_inst) {
    I.tma_g = -1;
    I.tma_z = 0;
  }
  if (c->opt.tile_loads == RT_LOADS_PLAIN || !encode_tiled()) return;
  std::vector<int> nx(c->n_dev), ny(c->n_dev);
  for (int d = 0; d < c->n_dev; ++d) {
    nx[d] = c->h_inst[d].nx;
    ny[d] = c->h_inst[d].ny;
  }
  const std::vector<rt::TmaRun> runs =
      rt::tma_plan(nx.data(), ny.data(), c->n_dev, c->esz, kTmaMinNx, kTmaMinNy, rt::TMA_GROUPS);
  const void* probe = reinterpret_cast<const void*>(uintptr_t(1) << 20);  // any 256-byte aligned address
  for (const rt::TmaRun& g : runs) {
    CUtensorMap m;
    bool ok = true;
    for (int rows : {kStageBoxRows[0], kStageBoxRows[1], kStageBoxRows[2], kAdjBoxRowsU[0], kAdjBoxRowsK[0],
                     kAdjBoxRowsU[1], kAdjBoxRowsK[1]})
      ok = ok && encode_group(c, g, probe, rows, &m);
    if (!ok) continue;
    const int gi = (int)c->tma_groups.size();
    c->tma_groups.push_back(g);
    for (int k = 0; k < g.count; ++k) {
      c->h_inst[g.first + k].tma_g = gi;
      c->h_inst[g.first + k].tma_z = k;
    }
  }
}

template <class T>
cudaError_t stage(rt_ctx* c, int st, int mode, const T* src, const T* base, T* dst, int n) {
  const int L = rt::tile_list_of(c->stage_variant);
  rt::TileMaps tm;
  cudaError_t e = tile_maps(c, src, kStageBoxRows[L], tm);
  if (e != cudaSuccess) return e;
  const int ev = timing_begin(c, st - 1);
  e = rt::launch_stage<T>(c->stage_variant, c->lim, st, mode, c->d_inst, c->d_strips, c->nstrips, c->d_tiles_h[L],
                          c->ntiles_h[L], src, base, dst, c->run, n, tm, c->stream);
  timing_end(c, ev);
  return e == cudaSuccess ? exchange(c, dst) : e;
}

template <class T>
cudaError_t adjoint(rt_ctx* c, const T* U, const T* K, double ks, const T* E, double es, T* out, int n) {
  const int a = c->adj_rows == 24 ? 1 : 0;
  rt::TileMaps tmu, tmk;
  cudaError_t e = tile_maps(c, U, kAdjBoxRowsU[a], tmu);
  if (e == cudaSuccess) e = tile_maps(c, K, kAdjBoxRowsK[a], tmk);
  if (e != cudaSuccess) return e;
  const int ev = timing_begin(c, 2);
  e = rt::launch_adjoint<T>(c->adj_rows, c->lim, c->d_inst, a ? c->d_tiles_a24 : c->d_tiles,
                            a ? c->ntiles_a24 : c->ntiles, U, K, ks, E, es, out, c->run, n, tmu, tmk, c->stream);
  timing_end(c, ev);
  return e == cudaSuccess ? exchange(c, out) : e;
}

// Steps per captured chunk of the time loop.
constexpr int kGraphChunk = 64;

// Run `enqueue` (a fixed sequence of launches) as a cached CUDA graph: the
// first call captures and instantiates it, later calls with the same key
// replay it. Sampled kernel timing bypasses the graphs.
template <class F>
rt_status run_graph(rt_ctx* c, const GraphKey& key, F&& enqueue) {
  if (!c->graphs || c->time_every > 0) return enqueue();
  auto it = c->gcache.find(key);
  if (it == c->gcache.end()) {
    const long long l0 = c->launches;
    long long k0[3];
    for (int k = 0; k < 3; ++k) k0[k] = c->kind_launches[k];
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const rt_status s = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != RT_OK) {
      if (e == cudaSuccess && g) cudaGraphDestroy(g);
      return s;
    }
    CU(e);
    GraphEntry ent;
    const cudaError_t ei = cudaGraphInstantiate(&ent.exec, g, 0);
    cudaGraphDestroy(g);
    CU(ei);
    ent.launches = c->launches - l0;
    for (int k = 0; k < 3; ++k) ent.kind_launches[k] = c->kind_launches[k] - k0[k];
    c->launches = l0;  // counted below, when the graph runs
    for (int k = 0; k < 3; ++k) c->kind_launches[k] = k0[k];
    it = c->gcache.emplace(key, ent).first;
  }
  CU(cudaGraphLaunch(it->second.exec, c->stream));
  c->launches += it->second.launches;
  for (int k = 0; k < 3; ++k) c->kind_launches[k] += it->second.kind_launches[k];
  return RT_OK;
}

// Order the context's stream after the caller's stream (device inputs the
// caller produced there are complete before the library reads them).
rt_status enter(rt_ctx* c) {
  CU(cudaEventRecord(c->ev_in, c->user_stream));
  CU(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  return RT_OK;
}

void reset_accounting(rt_ctx* c) {
  c->launches = 0;
  c->bad_instance = c->bad_step = -1;
  c->bad_cell = -1;
  for (int k = 0; k < 3; ++k) { c->kind_launches[k] = 0; c->kind_ms[k] = 0.0; c->kind_samples[k] = 0; }
  c->evused.clear();
  for (int k = 0; k < 3; ++k) c->kind_pairs[k] = 0;
}

// Called after the stream has drained: fold the sampled event pairs.
void collect_timing(rt_ctx* c) {
  for (auto& u : c->evused) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->evpool[u.second], c->evpool[u.second + 1]) == cudaSuccess) {
      c->kind_ms[u.first] += ms;
      c->kind_samples[u.first] += 1;
    }
  }
  c->evused.clear();
  for (int k = 0; k < 3; ++k) c->kind_pairs[k] = 0;
}

rt_status upload_inst(rt_ctx* c) {
  CU(cudaMemcpyAsync(c->d_inst, c->h_inst.data(), c->h_inst.size() * sizeof(InstDev), cudaMemcpyHostToDevice,
                     c->stream));
  return RT_OK;
}

rt_status ensure_pool(rt_ctx* c, size_t n) {
  while (c->pool.size() < n) {
    void* p = nullptr;
    if (cudaMalloc(&p, c->slot_bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, RT_ENOMEM, "cannot allocate checkpoint slot %zu (%zu bytes)", c->pool.size(), c->slot_bytes);
    }
    c->pool.push_back(p);
  }
  if ((int)n + 2 > c->tab_cap) {
    if (c->d_tab) cudaFree(c->d_tab);
    c->tab_cap = (int)n + 64;
    CU(cudaMalloc(&c->d_tab, c->tab_cap * sizeof(void*)));
  }
  return RT_OK;
}

rt_status ensure_pool1(rt_ctx* c, size_t n) {
  while (c->pool1.size() < n) {
    void* p = nullptr;
    if (cudaMalloc(&p, c->slot_bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, RT_ENOMEM, "cannot allocate stage-1 slot %zu (%zu bytes)", c->pool1.size(), c->slot_bytes);
    }
    c->pool1.push_back(p);
  }
  return RT_OK;
}

rt_status upload_tab(rt_ctx* c, const std::vector<void*>& tab) {
  if ((int)tab.size() > c->tab_cap) {
    if (c->d_tab) cudaFree(c->d_tab);
    c->tab_cap = (int)tab.size() + 64;
    CU(cudaMalloc(&c->d_tab, c->tab_cap * sizeof(void*)));
  }
  CU(cudaMemcpyAsync(c->d_tab, tab.data(), tab.size() * sizeof(void*), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));  // tab is a stack vector of the caller
  return RT_OK;
}

rt_status read_run(rt_ctx* c, std::vector<int>& nstep, std::vector<double>& t, std::vector<int>& status) {
  nstep.resize(c->n_inst);
  t.resize(c->n_inst);
  status.resize(c->n_inst);
  CU(cudaMemcpyAsync(nstep.data(), c->run.nstep, c->n_inst * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(t.data(), c->run.t, c->n_inst * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(status.data(), c->run.status, c->n_inst * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

// The first instance whose status word is set: RT_ETIMEOUT for a TMA wait
// that ran out, RT_ENONFINITE for a non-finite or non-positive state, whose
// cell and step (the stage-2 check of step nstep - 1 found it, and the step
// control stopped the instance there) are kept for rt_run_stats.
rt_status nonfinite(rt_ctx* c, const std::vector<int>& nstep, const std::vector<int>& status) {
  for (int i = 0; i < c->n_inst; ++i)
    if (status[i] == 2) {
      c->bad_instance = i;
      return fail(c, RT_ETIMEOUT, "instance %d: a TMA tile load did not complete within its wait limit", i);
    }
  for (int i = 0; i < c->n_inst; ++i)
    if (status[i] != 0) {
      long long cell = -1;
      cudaMemcpy(&cell, c->run.bad_cell + i, sizeof(long long), cudaMemcpyDeviceToHost);
      c->bad_instance = i;
      c->bad_cell = cell;
      c->bad_step = nstep[i] - 1;
      return fail(c, RT_ENONFINITE, "instance %d: non-positive density/pressure or NaN at cell %lld after step %d",
                  i, cell, c->bad_step);
    }
  return RT_OK;
}

// A failed call still reports where the state went bad.
rt_status failed_call(rt_ctx* c, rt_run_stats* st, rt_status s) {
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->bad_instance = c->bad_instance;
    st->bad_step = c->bad_step;
    st->bad_cell = c->bad_cell;
  }
  return s;
}

// Forward plan: kind 0 = ping-pong sA/sB; kind 1 = ping-pong plus a copy of
// every S-th state into pool[k]; kind 2 = every state n stored in pool[n];
// kind 3 = plain forward, then binomial (revolve) recomputation from U^0
// with `slots` checkpoint slots.
struct Plan {
  int kind = 0;
  int S = 0;
  int slots = 0;  // pool slots available to kind 2
};

// Inject v into the base state of every instance (k_inject), which also
// records dt of step 0. A fresh run (not a replay) first clears the dt
// records, so that steps no CTA reaches stay inactive.
template <class T>
rt_status inject(rt_ctx* c, const double* d_v, void* U0, bool replay = false) {
  if (!replay) {
    CU(cudaMemsetAsync(c->run.dtrec, 0, (size_t)c->n_inst * c->opt.max_steps * sizeof(double), c->stream));
    CU(cudaMemsetAsync(c->run.wrec, 0, (size_t)c->n_inst * c->opt.max_steps * sizeof(double), c->stream));
    CU(cudaMemsetAsync(c->run.dtc, 0, (size_t)c->n_inst * c->opt.max_steps * sizeof(rt::StepC<T>), c->stream));
  }
  CU(cudaMemsetAsync(c->run.wmin, 0xff, c->n_inst * sizeof(unsigned long long), c->stream));
  CU(cudaMemsetAsync(c->run.counter, 0, c->n_inst * sizeof(unsigned int), c->stream));
  CU(cudaMemsetAsync(c->run.status, 0, c->n_inst * sizeof(int), c->stream));
  CU(rt::launch_inject<T>(c->d_inst, c->d_tiles, c->ntiles, d_v, slotp<T>(U0), c->run, replay ? 0 : 1, c->stream));
  CU(exchange(c, U0));
  ++c->launches;
  return RT_OK;
}

// Estimated step count: fixed-step instances give theirs; horizon instances
// T / dt0, with dt0 the first step the inject kernel recorded.
rt_status estimate_steps(rt_ctx* c, int* n_est) {
  std::vector<double> dt0(c->n_inst);
  CU(cudaMemcpy2DAsync(dt0.data(), sizeof(double), c->run.dtrec, (size_t)c->opt.max_steps * sizeof(double),
                       sizeof(double), c->n_inst, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  long long best = 1;
  for (int i = 0; i < c->n_inst; ++i) {
    if (!c->h_inst[c->dev_first[i]].enabled) continue;
    const rt_problem& P = c->prob[i];
    if (P.nsteps > 0) { best = std::max<long long>(best, P.nsteps); continue; }
    if (!(dt0[i] > 0.0) || !(dt0[i] < kMaxFinite)) continue;
    best = std::max<long long>(best, (long long)std::ceil(P.T / dt0[i]));
  }
  *n_est = (int)std::min<long long>(best, c->opt.max_steps);
  return RT_OK;
}

bool all_done(rt_ctx* c, const std::vector<int>& nstep, const std::vector<double>& t, const std::vector<int>& status) {
  for (int i = 0; i < c->n_inst; ++i) {
    if (!c->h_inst[c->dev_first[i]].enabled || status[i] != 0) continue;
    const rt_problem& P = c->prob[i];
    if (P.nsteps > 0 ? nstep[i] < P.nsteps : t[i] < P.T) return false;
  }
  return true;
}

// March every instance from the injected state to its horizon. mode 0: CFL
// control; mode 1: replay the recorded dt sequence for `replay_steps` steps.
template <class T>
rt_status march(rt_ctx* c, const Plan& plan, int mode, int n_est, int replay_steps, int* n_done,
                int sample_every = 0, const std::function<rt_status(int)>* sampler = nullptr) {
  int n = 0;
  int target = mode == 1 ? replay_steps : n_est;
  const int smode = mode == 1 ? 1 : 0;
  std::vector<int> nstep, status;
  std::vector<double> t;
  auto steps = [&](int a, int b) -> rt_status {
    for (int k = a; k < b; ++k) {
      void *src, *dst, *u1 = c->sU1;
      if (plan.kind == 2) {
        src = c->pool[k];
        dst = c->pool[k + 1];
        u1 = c->pool1[k];
      } else {
        src = (k & 1) ? c->sB : c->sA;
        dst = (k & 1) ? c->sA : c->sB;
        if (plan.kind == 1 && k % plan.S == 0)
          CU(cudaMemcpyAsync(c->pool[plan.S + k / plan.S], src, c->slot_bytes, cudaMemcpyDeviceToDevice,
                             c->stream));
      }
      CU(stage<T>(c, 1, smode == 1 ? 2 : 0, slotp<T>(src), nullptr, slotp<T>(u1), k));
      CU(stage<T>(c, 2, smode, slotp<T>(u1), slotp<T>(src), slotp<T>(dst), k));
    }
    return RT_OK;
  };
  for (;;) {
    while (n < target) {
      int b = std::min(target, (n / kGraphChunk + 1) * kGraphChunk);
      if (sample_every > 0) b = std::min(b, (n / sample_every + 1) * sample_every);
      if (b > c->opt.max_steps) return fail(c, RT_EINVAL, "step limit %d reached", c->opt.max_steps);
      if (plan.kind == 2 && b >= plan.slots)
        return fail(c, RT_ENOMEM, "stored-state plan ran out of slots at step %d", b);
      if (plan.kind == 1) CHK(ensure_pool(c, plan.S + (b - 1) / plan.S + 1));  // no allocation inside a capture
      const GraphKey key{0, plan.kind, smode, c->stage_variant, c->lim, plan.S, n, b};
      CHK(run_graph(c, key, [&] { return steps(n, b); }));
      n = b;
      if (sampler && n % sample_every == 0) CHK((*sampler)(n));
    }
    CHK(read_run(c, nstep, t, status));
    CHK(nonfinite(c, nstep, status));
    if (mode == 1 || all_done(c, nstep, t, status)) break;
    target = n + std::max(16, n / 16);
  }
  *n_done = n;
  c->h_nstep = nstep;
  int mx = 0;
  for (int i = 0; i < c->n_inst; ++i) mx = std::max(mx, nstep[i]);
  c->last_steps = mx;
  c->last_kind = plan.kind == 2 ? 2 : 0;
  c->have_run = true;
  return RT_OK;
}

template <class T>
rt_status objective(rt_ctx* c, const Plan& plan, bool cotangent, double* ek_out) {
  std::vector<void*> tab;
  int mod;
  if (plan.kind == 2) {
    tab.assign(c->pool.begin(), c->pool.begin() + plan.slots);
    mod = 0;
  } else {
    tab = {c->sA, c->sB};
    mod = 2;
  }
  CHK(upload_tab(c, tab));
  CU(rt::launch_objective<T>(c->d_inst, c->d_tiles, c->ntiles, reinterpret_cast<T* const*>(c->d_tab), mod,
                             c->run.nstep, ek_out, cotangent ? slotp<T>(c->lA) : nullptr,
                             cotangent ? slotp<T>(c->lB) : nullptr, c->d_partials, c->stream));
  if (cotangent) {
    CU(exchange(c, c->lA));
    CU(exchange(c, c->lB));
  }
  CU(rt::launch_finalize(c->d_pinst, c->n_inst, c->d_partials, 2, 1, c->d_sums, c->stream));
  c->launches += 2;
  return RT_OK;
}

rt_status copy_in(rt_ctx* c, const double* v, int flags, double* dst) {
  const size_t bytes = c->total_v * sizeof(double);
  CU(cudaMemcpyAsync(dst, v, bytes, (flags & RT_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->stream));
  return RT_OK;
}

rt_status copy_out(rt_ctx* c, const double* src, int flags, double* out) {
  const size_t bytes = c->total_v * sizeof(double);
  CU(cudaMemcpyAsync(out, src, bytes, (flags & RT_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->stream));
  return RT_OK;
}

rt_status read_J(rt_ctx* c, double* J_out, double* J_ke_out) {
  std::vector<double> s(2 * c->n_inst);
  CU(cudaMemcpyAsync(s.data(), c->d_sums, s.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->n_inst; ++i) {
    if (J_out) J_out[i] = c->prob[i].objective == RT_OBJ_EK_ANOMALY_L2 ? s[2 * i + 1] : s[2 * i];
    if (J_ke_out) J_ke_out[i] = s[2 * i];
  }
  return RT_OK;
}

void fill_stats(rt_ctx* c, rt_run_stats* st, float ms, int segments) {
  if (!st) return;
  st->steps = c->last_steps;
  st->segments = segments;
  st->bad_instance = -1;
  st->bad_step = -1;
  st->bad_cell = -1;
  double cu = 0.0;
  for (int i = 0; i < c->n_inst; ++i) cu += (double)c->prob[i].nx * c->prob[i].ny * c->h_nstep[i];
  st->cell_updates = cu;
  st->ms = ms;
  st->launches = c->launches;
}

template <class T>
rt_status forward_impl(rt_ctx* c, const double* d_v, int flags, double* J_out, double* J_ke_out, int* steps) {
  const bool replay = (flags & RT_REPLAY_DT) != 0;
  if (replay && !c->have_run) return fail(c, RT_ESTATE, "RT_REPLAY_DT needs a previous run");
  const int replay_steps = c->last_steps;
  Plan plan;
  CHK(inject<T>(c, d_v, c->sA, replay));
  int n_est = replay_steps;
  if (!replay) CHK(estimate_steps(c, &n_est));
  int n_done = 0;
  CHK(march<T>(c, plan, replay ? 1 : 0, n_est, replay_steps, &n_done));
  CHK(objective<T>(c, plan, false, nullptr));
  CHK(read_J(c, J_out, J_ke_out));
  if (steps) *steps = n_done;
  return RT_OK;
}

// Forward run that samples t, KE and h_mix of every instance after step 0,
// every `every` steps and at the end (Sec. 4.3). samples receives one
// [n_inst][4] block {t, KE, h_mix, nstep} per sampling point; an instance that
// has reached its horizon repeats its final values, which the caller drops.
template <class T>
rt_status series_impl(rt_ctx* c, const double* d_v, int flags, int every, std::vector<double>& samples) {
  const bool replay = (flags & RT_REPLAY_DT) != 0;
  if (replay && !c->have_run) return fail(c, RT_ESTATE, "RT_REPLAY_DT needs a previous run");
  if (!c->d_rows) {
    std::vector<int2> rows;
    for (int i = 0; i < c->n_inst; ++i)
      for (int y = 0; y < c->prob[i].ny; ++y) rows.push_back(make_int2(i, y));
    c->total_rows = (int)rows.size();
    CU(cudaMalloc(&c->d_rows, rows.size() * sizeof(int2)));
    CU(cudaMalloc(&c->d_rowsum, rows.size() * sizeof(double2)));
    CU(cudaMalloc(&c->d_sample, (size_t)c->n_inst * 4 * sizeof(double)));
    CU(cudaMemcpyAsync(c->d_rows, rows.data(), rows.size() * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  const int replay_steps = c->last_steps;
  Plan plan;
  CHK(inject<T>(c, d_v, c->sA, replay));
  int n_est = replay_steps;
  if (!replay) CHK(estimate_steps(c, &n_est));
  std::function<rt_status(int)> take = [&](int) -> rt_status {
    const std::vector<void*> tab = {c->sA, c->sB};
    CHK(upload_tab(c, tab));
    CU(rt::launch_row_sums<T>(c->d_inst, c->d_rows, c->total_rows, reinterpret_cast<T* const*>(c->d_tab),
                              c->run.nstep, c->d_rowsum, c->stream));
    CU(rt::launch_series_sample(c->d_pinst, c->n_inst, c->d_rowsum, c->run.t, c->run.nstep, c->d_sample, c->stream));
    c->launches += 2;
    const size_t at = samples.size();
    samples.resize(at + 4 * c->n_inst);
    CU(cudaMemcpyAsync(samples.data() + at, c->d_sample, 4 * c->n_inst * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return RT_OK;
  };
  CHK(take(0));
  int n_done = 0;
  CHK(march<T>(c, plan, replay ? 1 : 0, n_est, replay_steps, &n_done, every, &take));
  return take(n_done);
}

// Binomial-checkpointing reverse sweep over steps [l, r) given U^l in `Ul`,
// with the checkpoint slots in `free` unused; the split points and the count
// of recomputed steps are those of rt_revolve.h (Griewank & Walther's
// optimum). Every step's adjoint needs U^n and its stage-1 state, recomputed
// from the nearest checkpoint.
template <class T>
struct Revolve {
  rt_ctx* c;
  std::vector<void*> free;  // unused checkpoint slots
  void* scratch[2];         // ping-pong for intermediate states while advancing
  void* leaf_state;         // target of the slot-free (quadratic) recomputation
  T* lam[2];
  T* l1;
  std::function<rt_status(int, T*, T*)> post;  // after each step's pull-back (n, U^n, U1), if set
  long long recomputed = 0;

  // advance U from step a (in src) to step b, result in dst; src and dst are
  // never scratch slots, intermediates alternate between the two scratch slots
  rt_status advance(int a, int b, void* src, void* dst) {
    void* cur = src;
    for (int k = a; k < b; ++k) {
      void* out = (k == b - 1) ? dst : (cur == scratch[0] ? scratch[1] : scratch[0]);
      CU(stage<T>(c, 1, 2, slotp<T>(cur), nullptr, slotp<T>(c->sU1), k));
      CU(stage<T>(c, 2, 2, slotp<T>(c->sU1), slotp<T>(cur), slotp<T>(out), k));
      cur = out;
      ++recomputed;
    }
    return RT_OK;
  }
  rt_status leaf(int n, void* Un) {
    CU(stage<T>(c, 1, 2, slotp<T>(Un), nullptr, slotp<T>(c->sU1), n));
    CU(adjoint<T>(c, slotp<T>(c->sU1), lam[(n + 1) & 1], 0.5, nullptr, 0.0, l1, n));
    CU(adjoint<T>(c, slotp<T>(Un), l1, 1.0, lam[(n + 1) & 1], 0.5, lam[n & 1], n));
    return post ? post(n, slotp<T>(Un), slotp<T>(c->sU1)) : RT_OK;
  }
  rt_status reverse(int l, int r, void* Ul) {
    const int n = r - l;
    if (n == 1) return leaf(l, Ul);
    const int s = (int)free.size();
    if (s == 0) {  // no slot left: recompute from l for every step
      for (int k = r - 1; k >= l; --k) {
        if (k == l) {
          CHK(leaf(l, Ul));
        } else {
          CHK(advance(l, k, Ul, leaf_state));
          CHK(leaf(k, leaf_state));
        }
      }
      return RT_OK;
    }
    const int m = l + rt::revolve_split(n, s);
    void* Um = free.back();
    free.pop_back();
    CHK(advance(l, m, Ul, Um));
    CHK(reverse(m, r, Um));
    free.push_back(Um);
    return reverse(l, m, Ul);
  }
};

// Gradient: forward with checkpoints, terminal cotangent, then for each step
// in reverse: recompute U1 = stage1(U^n), lam1 = (dStage2/dU1)^T lam^{n+1},
// lam^n = lam^{n+1}/2 + lam1 + (dL/dU^n)^T lam1 dt (SSP-RK2 transposed).
template <class T>
rt_status gradient_impl(rt_ctx* c, const double* d_v, double* J_out, double* d_g, int* segments_out,
                        bool dt_grad = false) {
  CHK(inject<T>(c, d_v, c->sA));
  int n_est = 1;
  CHK(estimate_steps(c, &n_est));
  Plan plan;
  const double need_all = (2.0 * ((double)n_est * 1.1 + 16.0)) * (double)c->slot_bytes;
  int mode = c->opt.ckpt;
  const double S_est = std::ceil(std::sqrt((double)n_est));
  const double need_sqrt = (2.0 * S_est + (double)n_est / S_est + 4.0) * (double)c->slot_bytes;
  if (mode == RT_CKPT_AUTO)
    mode = need_all <= c->mem_cap ? RT_CKPT_STORE_ALL : (need_sqrt <= c->mem_cap ? RT_CKPT_SQRT : RT_CKPT_REVOLVE);
  if (mode == RT_CKPT_REVOLVE) {
    plan.kind = 3;
    plan.slots = std::max(0, (int)(c->mem_cap / (double)c->slot_bytes) - 4);
    CHK(ensure_pool(c, plan.slots + 4));  // + U^0 slot, 2 scratch, 1 leaf state
  } else if (mode == RT_CKPT_STORE_ALL) {
    plan.kind = 2;
    plan.slots = (int)(n_est * 1.1 + 16);
    CHK(ensure_pool(c, plan.slots));
    CHK(ensure_pool1(c, plan.slots));
    CHK(inject<T>(c, d_v, c->pool[0]));
  } else {
    plan.kind = 1;
    plan.S = std::max(1, (int)std::ceil(std::sqrt((double)n_est)));
    CHK(ensure_pool(c, plan.S + n_est / plan.S + 2));
    CHK(ensure_pool1(c, plan.S));
  }
  int n_done = 0;
  Plan fplan = plan;
  if (plan.kind == 3) fplan = Plan();  // revolve: plain forward first, recomputation from U^0 later
  Range forward_range("forward sweep");
  rt_status s = march<T>(c, fplan, 0, n_est, 0, &n_done);
  if (s == RT_ENOMEM && plan.kind == 2) {  // the run outgrew the stored-state plan: redo it checkpointed
    plan = Plan();
    plan.kind = 1;
    plan.S = std::max(1, (int)std::ceil(std::sqrt((double)n_est * 1.5)));
    CHK(ensure_pool(c, plan.S + 2 * n_est / plan.S + 2));
    CHK(ensure_pool1(c, plan.S));
    CHK(inject<T>(c, d_v, c->sA));
    s = march<T>(c, plan, 0, n_est, 0, &n_done);
  }
  if (s != RT_OK) return s;
  CHK(objective<T>(c, fplan, true, nullptr));
  CHK(read_J(c, J_out, nullptr));
  forward_range.end();
  Range reverse_range("reverse sweep");
  const int N = c->last_steps;
  T* lam[2] = {slotp<T>(c->lA), slotp<T>(c->lB)};
  T* l1 = slotp<T>(c->l1);
  // lam1 = (dStage2/dU1)^T lam^{n+1};  lam^n = lam^{n+1}/2 + (dStage1/dU^n)^T lam1
  // With dt_grad, the step-control term of step n (after its frozen-dt
  // pull-back): U^{n+1} is recomputed into sA (free during the reverse
  // sweep), b_n = <lam^{n+1}, dU^{n+1}/d dt_n> is reduced per instance, and
  // lam^n gains the derivative of dt_n at the candidates of the minimum.
  auto dt_term = [&](int n, T* Un, T* U1) -> rt_status {
    if (!dt_grad) return RT_OK;
    CU(stage<T>(c, 2, 2, U1, Un, slotp<T>(c->sA), n));
    CU(rt::launch_dt_partials<T>(c->d_inst, c->d_tiles, c->ntiles, Un, U1, slotp<T>(c->sA), lam[(n + 1) & 1], l1,
                                 c->run, n, c->d_partials, c->stream));
    CU(rt::launch_dt_coef(c->d_pinst, c->n_inst, c->d_partials, c->run, n, c->d_blast, c->d_coef, c->stream));
    CU(rt::launch_dt_apply<T>(c->d_inst, c->d_tiles, c->ntiles, Un, lam[n & 1], c->run, n, c->d_coef, c->stream));
    CU(exchange(c, lam[n & 1]));
    c->launches += 3;
    return RT_OK;
  };
  if (dt_grad) CU(cudaMemsetAsync(c->d_blast, 0, c->n_inst * sizeof(double), c->stream));
  auto reverse_step = [&](int n, T* Un, T* U1) -> rt_status {
    CU(adjoint<T>(c, U1, lam[(n + 1) & 1], 0.5, nullptr, 0.0, l1, n));
    CU(adjoint<T>(c, Un, l1, 1.0, lam[(n + 1) & 1], 0.5, lam[n & 1], n));
    return dt_term(n, Un, U1);
  };
  int segments = 1;
  if (plan.kind == 3) {  // dynamic recursion: launched directly
    Revolve<T> rv;
    rv.c = c;
    for (int k = 0; k < plan.slots; ++k) rv.free.push_back(c->pool[4 + k]);
    rv.scratch[0] = c->pool[1];
    rv.scratch[1] = c->pool[2];
    rv.leaf_state = c->pool[3];
    rv.lam[0] = lam[0];
    rv.lam[1] = lam[1];
    rv.l1 = l1;
    rv.post = dt_term;
    CHK(inject<T>(c, d_v, c->pool[0], true));  // U^0 again; keeps the recorded dt sequence
    if (N > 0) CHK(rv.reverse(0, N, c->pool[0]));
    segments = -(int)std::min<long long>(rv.recomputed, 2000000000LL);  // reported as minus the recomputed steps
  } else if (plan.kind == 2) {
    for (int hi = N; hi > 0;) {
      const int lo = ((hi - 1) / kGraphChunk) * kGraphChunk;
      const GraphKey key{1, 2, dt_grad ? 1 : 0, c->stage_variant, c->lim, 0, lo, hi};
      CHK(run_graph(c, key, [&]() -> rt_status {
        for (int n = hi - 1; n >= lo; --n) CHK(reverse_step(n, slotp<T>(c->pool[n]), slotp<T>(c->pool1[n])));
        return RT_OK;
      }));
      hi = lo;
    }
  } else {
    const int S = plan.S;
    segments = (N + S - 1) / S;
    for (int k = segments - 1; k >= 0; --k) {
      Range segment_range("checkpoint segment: recompute and reverse");
      const int n0 = k * S, n1 = std::min(N, n0 + S);
      auto seg = [&](int n) -> T* { return n == n0 ? slotp<T>(c->pool[S + k]) : slotp<T>(c->pool[n - n0]); };
      auto seg1 = [&](int n) -> T* { return slotp<T>(c->pool1[n - n0]); };
      // recompute the segment from its checkpoint, keeping U^n and U1 of every step
      const GraphKey key{2, 1, dt_grad ? 1 : 0, c->stage_variant, c->lim, S, n0, n1};
      CHK(run_graph(c, key, [&]() -> rt_status {
        for (int n = n0; n < n1; ++n) {
          CU(stage<T>(c, 1, 2, seg(n), nullptr, seg1(n), n));
          if (n < n1 - 1) CU(stage<T>(c, 2, 2, seg1(n), seg(n), seg(n + 1), n));
        }
        for (int n = n1 - 1; n >= n0; --n) CHK(reverse_step(n, seg(n), seg1(n)));
        return RT_OK;
      }));
    }
  }
  CU(rt::launch_grad<T>(c->d_inst, c->d_tiles, c->ntiles, lam[0], d_v, d_g, c->stream));
  ++c->launches;
  if (segments_out) *segments_out = segments;
  {  // a tile load of the reverse sweep that gave up its wait (status 2)
    std::vector<int> nstep, status;
    std::vector<double> t;
    CHK(read_run(c, nstep, t, status));
    CHK(nonfinite(c, nstep, status));
  }
  return RT_OK;
}

rt_status field_sums(rt_ctx* c, int mode, const double* a, const double* b, std::vector<double>& out) {
  CU(rt::launch_field_reduce(mode, c->d_inst, c->d_tiles, c->ntiles, a, b, c->d_partials, c->stream));
  CU(rt::launch_finalize(c->d_pinst, c->n_inst, c->d_partials, 1, mode == 0 ? 1 : 0, c->d_sums, c->stream));
  out.resize(c->n_inst);
  CU(cudaMemcpyAsync(out.data(), c->d_sums, c->n_inst * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

// out = alpha_i a + beta_i b (b may be null)
rt_status axpby(rt_ctx* c, double* out, const std::vector<double>& alpha, const double* a,
                const std::vector<double>* beta, const double* b) {
  std::vector<double> sc(2 * c->n_inst, 0.0);
  for (int i = 0; i < c->n_inst; ++i) {
    sc[i] = alpha[i];
    if (beta) sc[c->n_inst + i] = (*beta)[i];
  }
  CU(cudaMemcpyAsync(c->d_scal, sc.data(), sc.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CU(rt::launch_field_axpby(c->d_inst, c->d_tiles, c->ntiles, out, c->d_scal, a, beta ? c->d_scal + c->n_inst : nullptr,
                            b, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

// Perturbation-sized fields, zeroed once when allocated: a CNOP search leaves
// the fields of a stopped instance untouched, and a zero coefficient on a
// never-written (zero) field keeps its iterate finite.
rt_status ensure_fields(rt_ctx* c, bool cnop) {
  const size_t bytes = c->total_v * sizeof(double);
  double** f[] = {&c->d_v, &c->d_g, &c->d_w1, &c->d_w2, &c->d_w3, &c->d_w4};
  for (int k = 0; k < (cnop ? 6 : 2); ++k)
    if (!*f[k]) {
      CU(cudaMalloc(f[k], bytes));
      CU(cudaMemsetAsync(*f[k], 0, bytes, c->stream));
    }
  return RT_OK;
}

rt_status set_enabled(rt_ctx* c, const std::vector<char>& en) {
  for (int i = 0; i < c->n_inst; ++i)
    for (int d = c->dev_first[i]; d < c->dev_first[i] + c->dev_count[i]; ++d) c->h_inst[d].enabled = en[i] ? 1 : 0;
  return upload_inst(c);
}

// Runs the baseline (v0 = 0) forward of every instance and keeps its final
// e_k as the reference field of the anomaly objective (Eq. objective).
template <class T>
rt_status baseline(rt_ctx* c) {
  CU(cudaMemsetAsync(c->d_v, 0, c->total_v * sizeof(double), c->stream));
  CU(cudaMalloc(&c->d_ek0, c->total_cells * sizeof(double)));
  Plan plan;
  CHK(inject<T>(c, c->d_v, c->sA));
  int n_est = 1;
  CHK(estimate_steps(c, &n_est));
  int n_done = 0;
  CHK(march<T>(c, plan, 0, n_est, 0, &n_done));
  CHK(objective<T>(c, plan, false, c->d_ek0));
  CU(cudaStreamSynchronize(c->stream));
  for (int d = 0; d < c->n_dev; ++d)
    c->h_inst[d].ek0 =
        c->prob[c->h_inst[d].run].objective == RT_OBJ_EK_ANOMALY_L2 ? c->d_ek0 + c->cell_off[d] : nullptr;
  CHK(upload_inst(c));
  c->have_run = false;
  return RT_OK;
}

// Autotuner: time a few CFL steps of the unperturbed batch with each
// stage-kernel variant and keep the faster (both give identical values).
template <class T>
rt_status autotune_stage(rt_ctx* c) {
  CU(cudaMemsetAsync(c->d_v, 0, c->total_v * sizeof(double), c->stream));
  const int variants[4] = {rt::STAGE_SWEEP, rt::STAGE_TILE8, rt::STAGE_TILE, rt::STAGE_TILE32};
  const int warm = 2, timed = 4;
  double best = 1e300;
  int best_v = rt::STAGE_SWEEP;
  for (int v : variants) {
    c->stage_variant = v;
    CHK(inject<T>(c, c->d_v, c->sA));
    for (int n = 0; n < warm + timed; ++n) {
      if (n == warm) CU(cudaEventRecord(c->ev0, c->stream));
      void* src = (n & 1) ? c->sB : c->sA;
      void* dst = (n & 1) ? c->sA : c->sB;
      CU(stage<T>(c, 1, 0, slotp<T>(src), nullptr, slotp<T>(c->sU1), n));
      CU(stage<T>(c, 2, 0, slotp<T>(c->sU1), slotp<T>(src), slotp<T>(dst), n));
    }
    CU(cudaEventRecord(c->ev1, c->stream));
    CU(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->tune_ms[v] = ms / timed;
    if (ms < best) { best = ms; best_v = v; }
  }
  c->stage_variant = best_v;
  c->have_run = false;
  return RT_OK;
}

// Adjoint autotuner (FP32): time three launches of the adjoint with 16- and
// 24-row tiles on the unperturbed batch at step 0 and keep the faster (both
// give the same values). RT_CNOP_ADJ_ROWS=16|24 fixes the choice instead.
template <class T>
rt_status autotune_adjoint(rt_ctx* c) {
  const char* f = getenv("RT_CNOP_ADJ_ROWS");
  if (f && (atoi(f) == 16 || atoi(f) == 24)) {
    c->adj_rows = sizeof(T) == 4 ? atoi(f) : 16;
    return RT_OK;
  }
  c->adj_rows = 16;
  if constexpr (sizeof(T) == 4) {
    CU(cudaMemsetAsync(c->d_v, 0, c->total_v * sizeof(double), c->stream));
    CHK(inject<T>(c, c->d_v, c->sA));
    CU(cudaMemsetAsync(c->lA, 0, c->slot_bytes, c->stream));
    const int reps = 3;
    double best = 1e300;
    int best_rows = 16;
    for (int k = 0; k < 2; ++k) {
      c->adj_rows = k ? 24 : 16;
      CU(adjoint<T>(c, slotp<T>(c->sA), slotp<T>(c->lA), 1.0, nullptr, 0.0, slotp<T>(c->lB), 0));  // warm-up
      CU(cudaEventRecord(c->ev0, c->stream));
      for (int r = 0; r < reps; ++r)
        CU(adjoint<T>(c, slotp<T>(c->sA), slotp<T>(c->lA), 1.0, nullptr, 0.0, slotp<T>(c->lB), 0));
      CU(cudaEventRecord(c->ev1, c->stream));
      CU(cudaEventSynchronize(c->ev1));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      c->adj_tune_ms[k] = ms / reps;
      if (ms < best) { best = ms; best_rows = c->adj_rows; }
    }
    c->adj_rows = best_rows;
    c->have_run = false;
  }
  return RT_OK;
}

struct Timer {
  rt_ctx* c;
  explicit Timer(rt_ctx* cc) : c(cc) { cudaEventRecord(c->ev0, c->stream); }
  float stop() {
    cudaEventRecord(c->ev1, c->stream);
    cudaEventSynchronize(c->ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    return ms;
  }
};

// ------------------------------------------------------------------ CNOP search
// Every instance switched back on when a CNOP search returns, on any path.
struct EnableAllOnExit {
  rt_ctx* c;
  ~EnableAllOnExit() {
    std::vector<char> en(c->n_inst, 1);
    set_enabled(c, en);
  }
};

// Start of a CNOP search (Sec. 3.4): v_inout into c->d_v, optionally
// localised at the interface, then scaled onto C = eps.
rt_status cnop_start(rt_ctx* c, const cnop_params* prm, const double* v_inout, int flags,
                     const std::vector<double>& eps) {
  const int N = c->n_inst;
  CHK(copy_in(c, v_inout, flags, c->d_v));
  if (prm->h_loc > 0.0) CU(rt::launch_localise(c->d_inst, c->d_tiles, c->ntiles, prm->h_loc, c->d_v, c->stream));
  std::vector<double> C, sc(N);
  CHK(field_sums(c, 0, c->d_v, nullptr, C));
  for (int i = 0; i < N; ++i) {
    if (!(C[i] > 0.0) || !std::isfinite(C[i]))
      return fail(c, RT_EINVAL, "start field of instance %d has C = %g (needs 0 < C < inf)", i, C[i]);
    sc[i] = std::sqrt(eps[i] / C[i]);
  }
  return axpby(c, c->d_v, sc, c->d_v, nullptr, nullptr);
}

// L-BFGS work fields: the (s, y) ring of m pairs plus the constraint normal.
rt_status ensure_pairs(rt_ctx* c, int m) {
  if (c->d_pairs && c->pairs_m >= m) return RT_OK;
  if (c->d_pairs) cudaFree(c->d_pairs);
  c->d_pairs = nullptr;
  c->pairs_m = 0;
  const size_t bytes = (size_t)(2 * m + 1) * c->total_v * sizeof(double);
  CU(cudaMalloc(&c->d_pairs, bytes));
  CU(cudaMemsetAsync(c->d_pairs, 0, bytes, c->stream));
  c->pairs_m = m;
  return RT_OK;
}

// max |a| per instance
rt_status field_max_abs(rt_ctx* c, const double* a, std::vector<double>& out) {
  CU(rt::launch_field_reduce(2, c->d_inst, c->d_tiles, c->ntiles, a, nullptr, c->d_partials, c->stream));
  CU(rt::launch_finalize_max(c->d_pinst, c->n_inst, c->d_partials, c->d_sums, c->stream));
  out.resize(c->n_inst);
  CU(cudaMemcpyAsync(out.data(), c->d_sums, c->n_inst * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

// Host side of a CNOP search: everything, besides the device fields v, g and
// the L-BFGS pair ring, that the iterations after k depend on. Kept whole so
// a run can be checkpointed and resumed.
struct CnopState {
  int k = 0, fevals = 0, gevals = 0, stored_iters = 0;
  std::vector<int> stop;                      // 0 running, 1 no acceptable step, 2 chi <= chi_tol
  std::vector<double> J, alpha, chi, gnorm;   // alpha: SPG step
  std::vector<std::vector<double>> hist;      // accepted J per instance
  std::vector<std::vector<double>> rho, gam;  // L-BFGS: [m][N]
};

const char kCkptMagic[8] = {'R', 'T', 'C', 'N', 'O', 'P', 'C', '1'};

// Checkpoint file: magic, sizes and method, eps, the host state, then the
// device fields v, g (and the L-BFGS ring) as FP64. Written to <path>.tmp and
// renamed, so a crash leaves the previous checkpoint intact.
rt_status save_checkpoint(rt_ctx* c, const char* path, int method, int m, const std::vector<double>& eps,
                          const CnopState& st) {
  const int N = c->n_inst;
  std::vector<double> field(c->total_v);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(c, RT_EIO, "cannot write checkpoint %s", tmp.c_str());
  bool ok = true;
  auto put = [&](const void* p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; };
  const long long hdr[9] = {N, (long long)c->total_v, method, m, (long long)c->esz, st.k, st.fevals, st.gevals,
                            st.stored_iters};
  put(kCkptMagic, sizeof(kCkptMagic));
  put(hdr, sizeof(hdr));
  put(eps.data(), N * sizeof(double));
  put(st.stop.data(), N * sizeof(int));
  put(st.J.data(), N * sizeof(double));
  put(st.alpha.data(), N * sizeof(double));
  put(st.chi.data(), N * sizeof(double));
  put(st.gnorm.data(), N * sizeof(double));
  for (int i = 0; i < N; ++i) {
    const long long n = (long long)st.hist[i].size();
    put(&n, sizeof(n));
    put(st.hist[i].data(), n * sizeof(double));
  }
  for (int j = 0; j < m; ++j) {
    put(st.rho[j].data(), N * sizeof(double));
    put(st.gam[j].data(), N * sizeof(double));
  }
  std::vector<const double*> dev = {c->d_v, c->d_g};
  for (int j = 0; j < 2 * m + 1 && method == RT_CNOP_LBFGS; ++j) dev.push_back(c->d_pairs + (size_t)j * c->total_v);
  for (const double* d : dev) {
    if (cudaMemcpyAsync(field.data(), d, c->total_v * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      fclose(f);
      return fail(c, RT_ECUDA, "checkpoint copy");
    }
    put(field.data(), c->total_v * sizeof(double));
  }
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) return fail(c, RT_EIO, "cannot write checkpoint %s", path);
  return RT_OK;
}

// Loads a checkpoint written by save_checkpoint for the same context,
// method, memory, precision and budgets. *found = false (and RT_OK) when the
// file does not exist.
rt_status load_checkpoint(rt_ctx* c, const char* path, int method, int m, const std::vector<double>& eps,
                          CnopState& st, bool* found) {
  const int N = c->n_inst;
  *found = false;
  FILE* f = fopen(path, "rb");
  if (!f) return RT_OK;
  *found = true;
  bool ok = true;
  auto get = [&](void* p, size_t n) { ok = ok && fread(p, 1, n, f) == n; };
  char magic[8];
  long long hdr[9];
  get(magic, sizeof(magic));
  get(hdr, sizeof(hdr));
  if (!ok || memcmp(magic, kCkptMagic, sizeof(magic)) != 0) {
    fclose(f);
    return fail(c, RT_EIO, "%s is not a CNOP checkpoint", path);
  }
  if (hdr[0] != N || hdr[1] != (long long)c->total_v || hdr[2] != method || hdr[3] != m || hdr[4] != (long long)c->esz) {
    fclose(f);
    return fail(c, RT_EINVAL, "checkpoint %s was written for another context, method, memory or precision", path);
  }
  std::vector<double> e(N);
  get(e.data(), N * sizeof(double));
  if (!ok || e != eps) {
    fclose(f);
    return fail(c, RT_EINVAL, "checkpoint %s was written for other budgets eps", path);
  }
  st.k = (int)hdr[5];
  st.fevals = (int)hdr[6];
  st.gevals = (int)hdr[7];
  st.stored_iters = (int)hdr[8];
  get(st.stop.data(), N * sizeof(int));
  get(st.J.data(), N * sizeof(double));
  get(st.alpha.data(), N * sizeof(double));
  get(st.chi.data(), N * sizeof(double));
  get(st.gnorm.data(), N * sizeof(double));
  for (int i = 0; i < N && ok; ++i) {
    long long n = 0;
    get(&n, sizeof(n));
    if (!ok || n < 0 || n > (1LL << 31)) { ok = false; break; }
    st.hist[i].resize(n);
    get(st.hist[i].data(), n * sizeof(double));
  }
  for (int j = 0; j < m; ++j) {
    get(st.rho[j].data(), N * sizeof(double));
    get(st.gam[j].data(), N * sizeof(double));
  }
  std::vector<double*> dev = {c->d_v, c->d_g};
  for (int j = 0; j < 2 * m + 1 && method == RT_CNOP_LBFGS; ++j) dev.push_back(c->d_pairs + (size_t)j * c->total_v);
  std::vector<double> field(c->total_v);
  for (double* d : dev) {
    get(field.data(), c->total_v * sizeof(double));
    if (!ok) break;
    if (cudaMemcpyAsync(d, field.data(), c->total_v * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      fclose(f);
      return fail(c, RT_ECUDA, "checkpoint copy");
    }
  }
  fclose(f);
  if (!ok) return fail(c, RT_EIO, "checkpoint %s is truncated", path);
  return RT_OK;
}

// The CNOP search of cnop_solve (Sec. 3.4, Eq. projection, App. A); the two
// methods' rules are stated at cnop_solve in the C header.
//
// Projected L-BFGS: on the budget surface C = eps the model gradient is that
// of J o P, gh = g - (<g, v> / <n, v>) n with n = dC/dv, and every direction
// is made tangent, p <- p - (<n, p> / <n, n>) n, so P puts each trial point
// back on the surface. The (s, y) pairs of the last m iterations live in a
// ring of device fields shared by all instances; an instance whose pair
// failed the curvature test, or that restarted, holds rho = 0 there, which
// makes the pair a no-op in the two-loop recursion (Nocedal & Wright
// Alg. 7.4).
//
// All instances advance in lockstep; dot products and the scalars of both
// methods are FP64, reduced per instance on the device.
template <class T>
rt_status cnop_run(rt_ctx* c, const cnop_params* prm, double* v_inout, int flags, double* J_out, cnop_result* res) {
  const int N = c->n_inst;
  const bool lbfgs = prm->method == RT_CNOP_LBFGS;
  const int m = lbfgs ? (prm->lbfgs_memory > 0 ? prm->lbfgs_memory : 10) : 0;
  std::vector<double> eps(prm->eps, prm->eps + N);
  for (int i = 0; i < N; ++i)
    if (!(eps[i] > 0.0) || !std::isfinite(eps[i])) return fail(c, RT_EINVAL, "eps[%d] must be positive", i);
  CHK(ensure_fields(c, true));
  if (lbfgs) CHK(ensure_pairs(c, m));
  EnableAllOnExit guard{c};
  std::vector<double> C, ones(N, 1.0), mones(N, -1.0), sc(N);
  double* v = c->d_v;
  double* g = c->d_g;  // dJ/dv at v (SPG) or the model gradient gh (L-BFGS)
  double* vt = c->d_w1;
  double* gt = c->d_w2;
  double* p = c->d_w3;  // search direction (L-BFGS p, SPG d); scratch once the step is taken
  double* tmp = c->d_w4;
  double* nrm = lbfgs ? c->d_pairs + (size_t)(2 * m) * c->total_v : nullptr;  // dC/dv at v
  auto S = [&](int j) { return c->d_pairs + (size_t)(2 * j) * c->total_v; };
  auto Y = [&](int j) { return c->d_pairs + (size_t)(2 * j + 1) * c->total_v; };
  const double amin = prm->alpha_min > 0 ? prm->alpha_min : 1e-30;
  const double amax = prm->alpha_max > 0 ? prm->alpha_max : 1e30;
  const int M = prm->gll_memory > 0 ? prm->gll_memory : 10;
  const int maxbt = prm->max_backtracks > 0 ? prm->max_backtracks : 30;

  CnopState st;
  st.stop.assign(N, 0);
  st.J.assign(N, 0.0);
  st.alpha.assign(N, 0.0);
  st.chi.assign(N, 0.0);
  st.gnorm.assign(N, 0.0);
  st.hist.assign(N, {});
  st.rho.assign(m, std::vector<double>(N, 0.0));
  st.gam.assign(m, std::vector<double>(N, 0.0));
  std::vector<char> on_surf(N, 0);
  auto running = [&](int i) { return st.stop[i] == 0; };
  auto set_running = [&]() -> rt_status {
    std::vector<char> e(N);
    for (int i = 0; i < N; ++i) e[i] = running(i);
    return set_enabled(c, e);
  };

  // chi = ||P(x + g) - x||_inf with g = dJ/dx (App. A), and ||g||; p is scratch
  auto stationarity = [&](const double* x, const double* gx) -> rt_status {
    std::vector<double> gg, chi;
    CHK(axpby(c, p, ones, x, &ones, gx));
    CHK(field_sums(c, 0, p, nullptr, C));
    for (int i = 0; i < N; ++i) sc[i] = C[i] <= eps[i] ? 1.0 : std::sqrt(eps[i] / C[i]);
    CHK(axpby(c, p, sc, p, nullptr, nullptr));
    CHK(axpby(c, p, ones, p, &mones, x));
    CHK(field_max_abs(c, p, chi));
    CHK(field_sums(c, 1, gx, gx, gg));
    for (int i = 0; i < N; ++i)
      if (running(i)) {
        st.chi[i] = chi[i];
        st.gnorm[i] = std::sqrt(gg[i]);
      }
    return RT_OK;
  };
  // on_surf[i] = C(x_i) >= eps (1 - 1e-10): x was put on the surface by P (up
  // to rounding). Then nrm = dC/dx and gx <- gx - (<gx, x> / <nrm, x>) nrm.
  auto model_gradient = [&](const double* x, double* gx) -> rt_status {
    CHK(field_sums(c, 0, x, nullptr, C));
    for (int i = 0; i < N; ++i) on_surf[i] = C[i] >= eps[i] * (1.0 - 1e-10);
    CU(rt::launch_field_weight(c->d_inst, c->d_tiles, c->ntiles, nrm, x, 0, c->stream));
    std::vector<double> gx_x, n_x, coef(N, 0.0);
    CHK(field_sums(c, 1, gx, x, gx_x));
    CHK(field_sums(c, 1, nrm, x, n_x));
    for (int i = 0; i < N; ++i)
      if (on_surf[i] && running(i)) coef[i] = -(gx_x[i] / n_x[i]);
    return axpby(c, gx, ones, gx, &coef, nrm);
  };
  // p <- p - (<nrm, p> / <nrm, nrm>) nrm for the instances flagged in `sel`
  auto tangent = [&](const std::vector<char>& sel) -> rt_status {
    std::vector<double> np_, nn, coef(N, 0.0);
    CHK(field_sums(c, 1, nrm, p, np_));
    CHK(field_sums(c, 1, nrm, nrm, nn));
    for (int i = 0; i < N; ++i)
      if (sel[i] && on_surf[i] && running(i)) coef[i] = -(np_[i] / nn[i]);
    return axpby(c, p, ones, p, &coef, nrm);
  };
  // SPG steps in the energy inner product <a, b>_E = sum rho0 a b dA of
  // Eq. constraint (<a, a>_E = 2 C(a)), in which the radial rescale P is the
  // exact projection onto the ball: its ascent direction is q = g / (rho0 dA),
  // the representer of g, so that its fixed points are the KKT points
  // g = lambda dC/dv. First step alpha = ||v||_E / ||q||_E; tmp is scratch.
  auto spg_alpha0 = [&]() -> rt_status {
    std::vector<double> cv, cq;
    CU(rt::launch_field_weight(c->d_inst, c->d_tiles, c->ntiles, tmp, g, 1, c->stream));
    CHK(field_sums(c, 0, v, nullptr, cv));
    CHK(field_sums(c, 0, tmp, nullptr, cq));
    for (int i = 0; i < N; ++i)
      st.alpha[i] = std::min(std::max(std::sqrt(cv[i]) / std::max(std::sqrt(cq[i]), 1e-300), amin), amax);
    return RT_OK;
  };

  FILE* log = nullptr;
  bool resumed = false;
  if (prm->resume && prm->checkpoint_path) CHK(load_checkpoint(c, prm->checkpoint_path, prm->method, m, eps, st, &resumed));
  if (prm->log_path) {
    log = fopen(prm->log_path, resumed ? "a" : "w");
    if (!log) return fail(c, RT_EIO, "cannot open log %s", prm->log_path);
    if (!resumed) fprintf(log, "# iter instance J C chi grad_norm lambda forward_evals gradient_evals\n");
  }
  struct CloseLog {
    FILE*& f;
    ~CloseLog() {
      if (f) fclose(f);
    }
  } close_log{log};
  auto record = [&](int iter, const std::vector<double>& lam) -> rt_status {
    if (res && res->J_history)
      for (int i = 0; i < N; ++i) res->J_history[(size_t)iter * N + i] = st.J[i];
    if (!log) return RT_OK;
    CHK(field_sums(c, 0, v, nullptr, C));
    for (int i = 0; i < N; ++i)
      fprintf(log, "%d %d %.17g %.17g %.17g %.17g %.17g %d %d\n", iter, i, st.J[i], C[i], st.chi[i], st.gnorm[i],
              lam.empty() ? 0.0 : lam[i], st.fevals, st.gevals);
    fflush(log);
    return RT_OK;
  };
  auto check_chi = [&]() {
    for (int i = 0; i < N; ++i)
      if (running(i) && prm->chi_tol > 0.0 && st.chi[i] <= prm->chi_tol) st.stop[i] = 2;
  };

  if (resumed) {
    if (lbfgs) {
      // on_surf and nrm at v, as the last model_gradient left them
      CHK(field_sums(c, 0, v, nullptr, C));
      for (int i = 0; i < N; ++i) on_surf[i] = C[i] >= eps[i] * (1.0 - 1e-10);
      CU(rt::launch_field_weight(c->d_inst, c->d_tiles, c->ntiles, nrm, v, 0, c->stream));
    }
  } else {
    CHK(cnop_start(c, prm, v_inout, flags, eps));
    CHK(set_running());
    CHK(gradient_impl<T>(c, v, st.J.data(), g, nullptr, (flags & RT_GRAD_DT) != 0));
    ++st.gevals;
    CHK(stationarity(v, g));
    if (lbfgs) CHK(model_gradient(v, g));
    else CHK(spg_alpha0());
    for (int i = 0; i < N; ++i) st.hist[i].push_back(st.J[i]);
    check_chi();
    CHK(record(0, {}));
  }

  auto slot = [&](int t) { return (st.stored_iters - 1 - t) % m; };  // t = 0: newest pair
  auto slot_used = [&](int j) {
    for (int i = 0; i < N; ++i)
      if (st.rho[j][i] != 0.0) return true;
    return false;
  };
  bool any_live = false;
  for (int i = 0; i < N; ++i) any_live = any_live || running(i);
  while (st.k < prm->max_iter && any_live) {
    Range iteration_range("cnop iteration");
    const int k = st.k;
    std::vector<double> gd, lam(N, 1.0), Jref(N), Jt(N), Jn(N);
    if (lbfgs) {
      // H0 = gamma I: <s,y>/<y,y> of the newest stored pair, else ||v|| / ||gh||
      const int npairs = std::min(st.stored_iters, m);
      std::vector<double> vv, gg, g0(N), gamma(N);
      std::vector<char> has_pair(N, 0), all(N, 1);
      CHK(field_sums(c, 1, v, v, vv));
      CHK(field_sums(c, 1, g, g, gg));
      for (int i = 0; i < N; ++i) {
        g0[i] = std::sqrt(vv[i]) / std::max(std::sqrt(gg[i]), 1e-300);
        gamma[i] = g0[i];
        for (int t = 0; t < npairs; ++t)
          if (st.rho[slot(t)][i] > 0.0) {
            gamma[i] = st.gam[slot(t)][i];
            has_pair[i] = 1;
            break;
          }
      }
      // two-loop recursion on p (starts as gh)
      std::vector<std::vector<double>> a(m, std::vector<double>(N, 0.0));
      CHK(axpby(c, p, ones, g, nullptr, nullptr));
      for (int t = 0; t < npairs; ++t) {
        const int j = slot(t);
        if (!slot_used(j)) continue;
        std::vector<double> sq, na(N);
        CHK(field_sums(c, 1, S(j), p, sq));
        for (int i = 0; i < N; ++i) {
          a[j][i] = st.rho[j][i] * sq[i];
          na[i] = -a[j][i];
        }
        CHK(axpby(c, p, ones, p, &na, Y(j)));
      }
      CHK(axpby(c, p, gamma, p, nullptr, nullptr));
      for (int t = npairs - 1; t >= 0; --t) {
        const int j = slot(t);
        if (!slot_used(j)) continue;
        std::vector<double> yr, coef(N);
        CHK(field_sums(c, 1, Y(j), p, yr));
        for (int i = 0; i < N; ++i) coef[i] = a[j][i] - st.rho[j][i] * yr[i];
        CHK(axpby(c, p, ones, p, &coef, S(j)));
      }
      CHK(tangent(all));
      // ascent check; a failed check drops the pairs and restarts from the
      // scaled model gradient
      std::vector<double> gp, keep(N, 1.0), gcoef(N, 0.0);
      CHK(field_sums(c, 1, g, p, gp));
      std::vector<char> restart(N, 0);
      bool any_restart = false;
      for (int i = 0; i < N; ++i)
        if (running(i) && has_pair[i] && gp[i] <= 0.0) {
          restart[i] = 1;
          any_restart = true;
          keep[i] = 0.0;
          gcoef[i] = g0[i];
          for (int j = 0; j < m; ++j) st.rho[j][i] = 0.0;
        }
      if (any_restart) {
        CHK(axpby(c, p, keep, p, &gcoef, g));
        CHK(tangent(restart));
      }
    } else {
      // d = P(v + alpha q) - v, q = g / (rho0 dA), and <g, d>
      CU(rt::launch_field_weight(c->d_inst, c->d_tiles, c->ntiles, tmp, g, 1, c->stream));
      CHK(axpby(c, vt, ones, v, &st.alpha, tmp));
      CHK(field_sums(c, 0, vt, nullptr, C));
      for (int i = 0; i < N; ++i) sc[i] = C[i] <= eps[i] ? 1.0 : std::sqrt(eps[i] / C[i]);
      CHK(axpby(c, vt, sc, vt, nullptr, nullptr));
      CHK(axpby(c, p, ones, vt, &mones, v));
      CHK(field_sums(c, 1, g, p, gd));
    }
    // trial point for the step lam and its sufficient-increase term: L-BFGS
    // vt = P(v + lam p), c <gh, vt - v>; SPG vt = v + lam d, c lam <g, d>.
    // Stopped instances keep vt = v.
    std::vector<double> term(N);
    auto trial = [&]() -> rt_status {
      CHK(axpby(c, vt, ones, v, &lam, p));
      if (!lbfgs) {
        for (int i = 0; i < N; ++i) term[i] = prm->armijo_c * lam[i] * gd[i];
        return RT_OK;
      }
      std::vector<double> gs;
      CHK(field_sums(c, 0, vt, nullptr, C));
      for (int i = 0; i < N; ++i) sc[i] = (!running(i) || C[i] <= eps[i]) ? 1.0 : std::sqrt(eps[i] / C[i]);
      CHK(axpby(c, vt, sc, vt, nullptr, nullptr));
      CHK(axpby(c, tmp, ones, vt, &mones, v));
      CHK(field_sums(c, 1, g, tmp, gs));
      for (int i = 0; i < N; ++i) term[i] = prm->armijo_c * gs[i];
      return RT_OK;
    };
    // non-monotone reference (Grippo, Lampariello & Lucidi, for the maximised
    // J): the worst, i.e. smallest, of the last M accepted values, so that J may
    // dip temporarily
    for (int i = 0; i < N; ++i) {
      const size_t h0 = st.hist[i].size() > (size_t)M ? st.hist[i].size() - M : 0;
      Jref[i] = *std::min_element(st.hist[i].begin() + h0, st.hist[i].end());
    }
    std::vector<char> acc(N, 0);
    for (int i = 0; i < N; ++i) acc[i] = !running(i);
    for (int bt = 0; bt < maxbt; ++bt) {
      CHK(trial());
      std::vector<char> e(N);
      for (int i = 0; i < N; ++i) e[i] = !acc[i];
      CHK(set_enabled(c, e));
      int steps = 0;
      CHK(forward_impl<T>(c, vt, RT_DEVICE_PTRS, Jt.data(), nullptr, &steps));
      ++st.fevals;
      bool all = true;
      for (int i = 0; i < N; ++i) {
        if (acc[i]) continue;
        if (Jt[i] >= Jref[i] + term[i]) acc[i] = 1;
        else { lam[i] *= 0.5; all = false; }
      }
      if (all) break;
    }
    for (int i = 0; i < N; ++i)
      if (!acc[i]) st.stop[i] = 1;
    for (int i = 0; i < N; ++i)
      if (!running(i)) lam[i] = 0.0;
    CHK(trial());  // the accepted point (v itself for stopped instances)
    any_live = false;
    for (int i = 0; i < N; ++i) any_live = any_live || running(i);
    if (!any_live) break;
    CHK(set_running());
    CHK(gradient_impl<T>(c, vt, Jn.data(), gt, nullptr, (flags & RT_GRAD_DT) != 0));
    ++st.gevals;
    CHK(stationarity(vt, gt));
    CHK(axpby(c, tmp, ones, vt, &mones, v));  // s = vt - v
    if (lbfgs) {
      CHK(model_gradient(vt, gt));
      // new pair: s, y = -(gh_new - gh) = gh - gh_new
      const int h = st.stored_iters % m;
      CHK(axpby(c, S(h), ones, tmp, nullptr, nullptr));
      CHK(axpby(c, Y(h), ones, g, &mones, gt));
      std::vector<double> sy, yy;
      CHK(field_sums(c, 1, S(h), Y(h), sy));
      CHK(field_sums(c, 1, Y(h), Y(h), yy));
      for (int i = 0; i < N; ++i) {
        const bool ok = running(i) && sy[i] > 0.0;
        st.rho[h][i] = ok ? 1.0 / sy[i] : 0.0;
        st.gam[h][i] = ok ? sy[i] / yy[i] : 0.0;
      }
      ++st.stored_iters;
    } else {
      // alpha = <s,s>_E / <s,y'>, y' = -(g_new - g), <s,s>_E = 2 C(s)
      std::vector<double> cs, sg, sgt;
      CHK(field_sums(c, 0, tmp, nullptr, cs));
      CHK(field_sums(c, 1, tmp, g, sg));
      CHK(field_sums(c, 1, tmp, gt, sgt));
      for (int i = 0; i < N; ++i) {
        if (!running(i)) continue;
        const double sy = sg[i] - sgt[i];
        st.alpha[i] = sy <= 0.0 ? amax : std::min(std::max(2.0 * cs[i] / sy, amin), amax);
      }
    }
    for (int i = 0; i < N; ++i) {
      if (!running(i)) continue;
      st.J[i] = Jn[i];
      st.hist[i].push_back(st.J[i]);
    }
    std::swap(c->d_v, c->d_w1);  // v <- vt
    std::swap(c->d_g, c->d_w2);  // g <- g_new
    v = c->d_v;
    g = c->d_g;
    vt = c->d_w1;
    gt = c->d_w2;
    st.k = k + 1;
    check_chi();
    CHK(record(st.k, lam));
    any_live = false;
    for (int i = 0; i < N; ++i) any_live = any_live || running(i);
    if (prm->checkpoint_path && prm->checkpoint_every > 0 && st.k % prm->checkpoint_every == 0)
      CHK(save_checkpoint(c, prm->checkpoint_path, prm->method, m, eps, st));
  }
  if (prm->checkpoint_path) CHK(save_checkpoint(c, prm->checkpoint_path, prm->method, m, eps, st));
  CHK(copy_out(c, v, flags, v_inout));
  CU(cudaStreamSynchronize(c->stream));
  if (J_out)
    for (int i = 0; i < N; ++i) J_out[i] = st.J[i];
  bool any_stuck = false;
  for (int i = 0; i < N; ++i) any_stuck = any_stuck || st.stop[i] == 1;
  if (res) {
    res->iterations = st.k;
    res->forward_evals = st.fevals;
    res->gradient_evals = st.gevals;
    std::vector<double> Cf;
    if (res->C) CHK(field_sums(c, 0, v, nullptr, Cf));
    for (int i = 0; i < N; ++i) {
      if (res->C) res->C[i] = Cf[i];
      if (res->chi) res->chi[i] = st.chi[i];
      if (res->grad_norm) res->grad_norm[i] = st.gnorm[i];
      if (res->stop) res->stop[i] = st.stop[i];
    }
  }
  if (any_stuck) return fail(c, RT_ENOTCONVERGED, "an instance found no acceptable step");
  return RT_OK;
}

}  // namespace

// =================================================================== C ABI
// ---------------------------------------------- spectra and reduced seeds
namespace {
// Work buffers of one spectral analysis, sized for the largest instance.
struct SpecWork {
  double2* a = nullptr;
  double2* b = nullptr;
  double* E = nullptr;
  unsigned char* keep = nullptr;
  int* ints = nullptr;   // [0] y_peak, [1] kept modes
  double* dbl = nullptr; // [0] total energy
  ~SpecWork() {
    cudaFree(a);
    cudaFree(b);
    cudaFree(E);
    cudaFree(keep);
    cudaFree(ints);
    cudaFree(dbl);
  }
};

rt_status spec_alloc(rt_ctx* c, SpecWork& w) {
  long long n = 0;
  for (const rt_problem& P : c->prob) {
    if (P.nx > rt::SPEC_MAX_N || P.ny > rt::SPEC_MAX_N)
      return fail(c, RT_EINVAL, "spectra need nx, ny <= %d", rt::SPEC_MAX_N);
    n = std::max(n, (long long)P.nx * P.ny);
  }
  CU(cudaMalloc(&w.a, n * sizeof(double2)));
  CU(cudaMalloc(&w.b, n * sizeof(double2)));
  CU(cudaMalloc(&w.E, n * sizeof(double)));
  CU(cudaMalloc(&w.keep, n));
  CU(cudaMalloc(&w.ints, 2 * sizeof(int)));
  CU(cudaMalloc(&w.dbl, sizeof(double)));
  CU(rt::spec_configure());
  return RT_OK;
}

// u_y of instance i: the last perturbed component of v
const double* uy_plane(rt_ctx* c, const double* v, int i) {
  const rt_problem& P = c->prob[i];
  return v + c->v_off[i] + (size_t)(P.perturb_ncomp - 1) * P.nx * P.ny;
}
}  // namespace

extern "C" {

rt_status rt_init(const rt_problem* problems, int n_instances, const rt_options* opt, void* cuda_stream,
                  rt_ctx** out) {
  if (!out) return RT_EINVAL;
  *out = nullptr;
  if (!problems || n_instances <= 0) return RT_EINVAL;
  Range range("rt_init");
  rt_ctx* c = new (std::nothrow) rt_ctx();
  if (!c) return RT_ENOMEM;
  auto bail = [&](rt_status s) {
    // keep the message readable for a caller that only sees the status
    fprintf(stderr, "rt_init: %s\n", c->err.c_str());
    rt_destroy(c);
    return s;
  };
  c->n_inst = n_instances;
  if (opt) c->opt = *opt;
  if (c->opt.max_steps <= 0) c->opt.max_steps = 200000;
  if (c->opt.precision != RT_FP64 && c->opt.precision != RT_FP32_STATE) {
    fail(c, RT_EINVAL, "precision");
    return bail(RT_EINVAL);
  }
  if (c->opt.tile_loads != RT_LOADS_TMA && c->opt.tile_loads != RT_LOADS_PLAIN) {
    fail(c, RT_EINVAL, "tile_loads must be RT_LOADS_TMA or RT_LOADS_PLAIN");
    return bail(RT_EINVAL);
  }
  c->esz = c->opt.precision == RT_FP64 ? sizeof(double) : sizeof(float);
  c->user_stream = static_cast<cudaStream_t>(cuda_stream);
  c->prob.assign(problems, problems + n_instances);
  for (int i = 0; i < n_instances; ++i) {
    rt_status s = validate(c, c->prob[i], i);
    if (s != RT_OK) return bail(s);
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    fail(c, RT_ECUDA, "no CUDA device");
    return bail(RT_ECUDA);
  }
  // instance layout, tiles, base state. A problem split into y-slabs gets one
  // device instance per slab: owned rows as even as possible (the first
  // ny % k slabs one row taller), plus kSlabHalo halo rows on each side
  // with a neighbouring slab.
  const int nslab = c->opt.y_slabs > 1 ? c->opt.y_slabs : 1;
  if (n_instances >= (1 << 24)) {  // tile descriptors carry the problem index in 24 bits
    fail(c, RT_EINVAL, "at most %d instances", (1 << 24) - 1);
    return bail(RT_EINVAL);
  }
  for (int i = 0; i < n_instances; ++i)
    if (nslab > 1 && c->prob[i].ny < kSlabHalo * nslab) {
      fail(c, RT_EINVAL, "instance %d: %d rows cannot give %d slabs of at least %d rows", i, c->prob[i].ny, nslab,
           kSlabHalo);
      return bail(RT_EINVAL);
    }
  c->v_off.resize(n_instances);
  c->dev_first.resize(n_instances);
  c->dev_count.assign(n_instances, nslab);
  long long cells = 0, voff = 0, rows = 0;
  for (int i = 0; i < n_instances; ++i) {
    const rt_problem& P = c->prob[i];
    c->v_off[i] = voff;
    voff += (long long)P.perturb_ncomp * P.nx * P.ny;
    rows += P.ny;
  }
  c->total_v = (size_t)voff;
  std::vector<double> base(2 * rows);
  long long roff = 0;
  for (int i = 0; i < n_instances; ++i) {
    const rt_problem& P = c->prob[i];
    std::vector<double> r, p;
    base_state(P, r, p);
    std::copy(r.begin(), r.end(), base.begin() + roff);
    std::copy(p.begin(), p.end(), base.begin() + rows + roff);
    c->dev_first[i] = (int)c->h_inst.size();
    const int tiles0 = (int)c->h_tiles.size(), strips0 = (int)c->h_strips.size();
    const int t8 = (int)c->h_tiles_h[0].size(), t32 = (int)c->h_tiles_h[2].size();
    const int hb = P.ny / nslab, extra = P.ny % nslab;
    int y0s = 0;
    for (int sl = 0; sl < nslab; ++sl) {
      const int y1s = y0s + hb + (sl < extra ? 1 : 0);
      const int e0 = sl > 0 ? y0s - kSlabHalo : y0s;
      const int e1 = sl < nslab - 1 ? y1s + kSlabHalo : y1s;
      InstDev I{};
      I.nx = P.nx;
      I.ny = e1 - e0;
      I.run = i;
      I.own0 = y0s - e0;
      I.own1 = y1s - e0;
      I.v_plane = (long long)P.nx * P.ny;
      I.bc_y = P.bc_y;
      I.limiter = P.limiter;
      I.nsteps = P.nsteps;
      I.ncomp = P.perturb_ncomp;
      I.objective = P.objective;
      I.enabled = 1;
      I.cell_off = cells;
      I.v_off = c->v_off[i] + (long long)y0s * P.nx;
      I.dx = (P.x1 - P.x0) / P.nx;
      I.dy = (P.y1 - P.y0) / P.ny;
      I.dA = I.dx * I.dy;
      I.y0 = P.y0 + e0 * I.dy;
      I.y_int = P.y_int;
      I.rho_l = P.rho_light;
      I.rho_h = P.rho_heavy;
      I.row_off = roff + e0;
      I.gamma = P.gamma;
      I.gm1 = P.gamma - 1.0;
      I.g_y = P.g_y;
      I.cfl = P.cfl;
      I.T = P.T;
      I.gamma_f = (float)I.gamma;
      I.gm1_f = (float)I.gm1;
      I.g_f = (float)I.g_y;
      I.dx_f = (float)I.dx;
      I.dy_f = (float)I.dy;
      I.flux = P.flux;
      I.flux_theta = P.flux == RT_FLUX_HYBRID ? P.flux_theta : 0.0;
      I.flux_theta_f = (float)I.flux_theta;
      const int d = (int)c->h_inst.size();
      I.tile_begin = (int)c->h_tiles.size();
      for (int ty = I.own0; ty < I.own1; ty += rt::TILE_Y)
        for (int x0 = 0; x0 < P.nx; x0 += rt::TILE_X)
          c->h_tiles.push_back(make_int4(d, x0, ty, i | (std::min(rt::TILE_Y, I.own1 - ty) << 24)));
      I.tile_end = (int)c->h_tiles.size();
      for (int ty = I.own0; ty < I.own1; ty += 24)  // the adjoint list of 24-row tiles
        for (int x0 = 0; x0 < P.nx; x0 += rt::TILE_X)
          c->h_tiles_a24.push_back(make_int4(d, x0, ty, i | (std::min(24, I.own1 - ty) << 24)));
      for (int L : {0, 2}) {  // the tile-stage lists of 8 and 32 rows
        const int h = L == 0 ? 8 : 32;
        for (int ty = I.own0; ty < I.own1; ty += h)
          for (int x0 = 0; x0 < P.nx; x0 += rt::TILE_X)
            c->h_tiles_h[L].push_back(make_int4(d, x0, ty, i | (std::min(h, I.own1 - ty) << 24)));
      }
      I.strip_begin = (int)c->h_strips.size();
      for (int ty = I.own0; ty < I.own1; ty += rt::STRIP_H)
        for (int x0 = 0; x0 < P.nx; x0 += rt::STRIP_W)
          c->h_strips.push_back(make_int4(d, x0, ty, i | (std::min(rt::STRIP_H, I.own1 - ty) << 24)));
      I.strip_end = (int)c->h_strips.size();
      I.ek0 = nullptr;
      c->cell_off.push_back(cells);
      cells += (long long)I.nx * I.ny;
      if (sl > 0) {  // halos between this slab and the one below
        const InstDev& L = c->h_inst.back();
        // this slab's lower halo rows <- the top owned rows of the slab below
        c->halos.push_back({I.cell_off, L.cell_off, (long long)I.nx * I.ny, (long long)L.nx * L.ny, 0,
                            L.own1 - kSlabHalo, P.nx});
        // the lower slab's upper halo rows <- this slab's bottom owned rows
        c->halos.push_back({L.cell_off, I.cell_off, (long long)L.nx * L.ny, (long long)I.nx * I.ny, L.own1,
                            I.own0, P.nx});
      }
      c->h_inst.push_back(I);
      y0s = y1s;
    }
    const int ntile_run = (int)c->h_tiles.size() - tiles0, nstrip_run = (int)c->h_strips.size() - strips0;
    for (int d = c->dev_first[i]; d < (int)c->h_inst.size(); ++d) {
      c->h_inst[d].run_tiles = ntile_run;
      c->h_inst[d].run_strips = nstrip_run;
      c->h_inst[d].run_tiles_h[0] = (int)c->h_tiles_h[0].size() - t8;
      c->h_inst[d].run_tiles_h[1] = ntile_run;
      c->h_inst[d].run_tiles_h[2] = (int)c->h_tiles_h[2].size() - t32;
    }
    roff += P.ny;
  }
  c->n_dev = (int)c->h_inst.size();
  c->total_cells = cells;
  c->slot_bytes = (size_t)(4 * cells) * c->esz;
  c->ntiles = (int)c->h_tiles.size();
  c->nstrips = (int)c->h_strips.size();
  c->lim = c->prob[0].limiter;
  for (int i = 1; i < n_instances; ++i)
    if (c->prob[i].limiter != c->lim) c->lim = -1;
  if (c->lim != RT_LIM_MINMOD) c->lim = -1;  // only minmod has specialised kernels
  for (int i = 0; i < n_instances; ++i)      // ... and only with the HLLC flux
    if (c->prob[i].flux != RT_FLUX_HLLC) c->lim = -1;
  const int N = n_instances;
#define INIT_CU(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      fail(c, e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA, "%s: %s", #call,           \
           cudaGetErrorString(e_));                                                              \
      return bail(e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA);                       \
    }                                                                                            \
  } while (0)
  INIT_CU(cudaMalloc(&c->d_base, base.size() * sizeof(double)));
  INIT_CU(cudaMemcpy(c->d_base, base.data(), base.size() * sizeof(double), cudaMemcpyHostToDevice));
  c->h_base_f.assign(base.begin(), base.end());
  c->base_rows = rows;
  INIT_CU(cudaMalloc(&c->d_base_f, base.size() * sizeof(float)));
  INIT_CU(cudaMemcpy(c->d_base_f, c->h_base_f.data(), base.size() * sizeof(float), cudaMemcpyHostToDevice));
  roff = 0;
  c->row_off.resize(N);
  for (int i = 0; i < N; ++i) {
    c->row_off[i] = roff;
    roff += c->prob[i].ny;
  }
  for (InstDev& I : c->h_inst) {  // row_off of a slab already includes its first held row
    I.rho0 = c->d_base + I.row_off;
    I.p0 = c->d_base + rows + I.row_off;
    I.rho0_f = c->d_base_f + I.row_off;
    I.p0_f = c->d_base_f + rows + I.row_off;
  }
  assign_tma_groups(c);
  INIT_CU(cudaMalloc(&c->d_inst, c->n_dev * sizeof(InstDev)));
  INIT_CU(cudaMemcpy(c->d_inst, c->h_inst.data(), c->n_dev * sizeof(InstDev), cudaMemcpyHostToDevice));
  if (nslab == 1) {
    c->d_pinst = c->d_inst;
  } else {  // one entry per problem whose tile range spans all its slabs
    std::vector<InstDev> pin(N);
    for (int i = 0; i < N; ++i) {
      const InstDev& F = c->h_inst[c->dev_first[i]];
      const InstDev& Lst = c->h_inst[c->dev_first[i] + c->dev_count[i] - 1];
      pin[i] = F;
      pin[i].tile_end = Lst.tile_end;
      pin[i].strip_end = Lst.strip_end;
      pin[i].ny = c->prob[i].ny;
      pin[i].own0 = 0;
      pin[i].own1 = c->prob[i].ny;
      pin[i].row_off = c->row_off[i];
    }
    INIT_CU(cudaMalloc(&c->d_pinst, N * sizeof(InstDev)));
    INIT_CU(cudaMemcpy(c->d_pinst, pin.data(), N * sizeof(InstDev), cudaMemcpyHostToDevice));
  }
  INIT_CU(cudaMalloc(&c->d_tiles, c->ntiles * sizeof(int4)));
  INIT_CU(cudaMemcpy(c->d_tiles, c->h_tiles.data(), c->ntiles * sizeof(int4), cudaMemcpyHostToDevice));
  c->h_tiles_h[1] = c->h_tiles;
  c->d_tiles_h[1] = c->d_tiles;
  c->ntiles_h[1] = c->ntiles;
  for (int L : {0, 2}) {
    c->ntiles_h[L] = (int)c->h_tiles_h[L].size();
    INIT_CU(cudaMalloc(&c->d_tiles_h[L], c->ntiles_h[L] * sizeof(int4)));
    INIT_CU(cudaMemcpy(c->d_tiles_h[L], c->h_tiles_h[L].data(), c->ntiles_h[L] * sizeof(int4),
                       cudaMemcpyHostToDevice));
  }
  c->ntiles_a24 = (int)c->h_tiles_a24.size();
  INIT_CU(cudaMalloc(&c->d_tiles_a24, c->ntiles_a24 * sizeof(int4)));
  INIT_CU(cudaMemcpy(c->d_tiles_a24, c->h_tiles_a24.data(), c->ntiles_a24 * sizeof(int4), cudaMemcpyHostToDevice));
  INIT_CU(cudaMalloc(&c->d_strips, c->nstrips * sizeof(int4)));
  INIT_CU(cudaMemcpy(c->d_strips, c->h_strips.data(), c->nstrips * sizeof(int4), cudaMemcpyHostToDevice));
  void** bufs[6] = {&c->sA, &c->sB, &c->sU1, &c->lA, &c->lB, &c->l1};
  for (void** b : bufs) INIT_CU(cudaMalloc(b, c->slot_bytes));
  c->run.n_inst = N;
  c->run.max_steps = c->opt.max_steps;
  INIT_CU(cudaMalloc(&c->run.dtrec, (size_t)N * c->opt.max_steps * sizeof(double)));
  INIT_CU(cudaMalloc(&c->run.wrec, (size_t)N * c->opt.max_steps * sizeof(double)));
  INIT_CU(cudaMemset(c->run.wrec, 0, (size_t)N * c->opt.max_steps * sizeof(double)));
  INIT_CU(cudaMalloc(&c->d_blast, (size_t)N * sizeof(double)));
  INIT_CU(cudaMalloc(&c->d_coef, (size_t)N * sizeof(double)));
  INIT_CU(cudaMalloc(&c->run.t, N * sizeof(double)));
  INIT_CU(cudaMalloc(&c->run.nstep, N * sizeof(int)));
  INIT_CU(cudaMalloc(&c->run.wmin, N * sizeof(unsigned long long)));
  INIT_CU(cudaMalloc(&c->run.counter, N * sizeof(unsigned int)));
  INIT_CU(cudaMalloc(&c->run.dtc, (size_t)N * c->opt.max_steps * 4 * c->esz));
  INIT_CU(cudaMemset(c->run.dtc, 0, (size_t)N * c->opt.max_steps * 4 * c->esz));
  INIT_CU(cudaMemset(c->run.dtrec, 0, (size_t)N * c->opt.max_steps * sizeof(double)));
  INIT_CU(cudaMalloc(&c->run.status, N * sizeof(int)));
  INIT_CU(cudaMalloc(&c->run.bad_cell, N * sizeof(long long)));
  INIT_CU(cudaMalloc(&c->d_partials, (size_t)c->ntiles * 2 * sizeof(double)));
  INIT_CU(cudaMalloc(&c->d_sums, (size_t)N * 2 * sizeof(double)));
  INIT_CU(cudaMalloc(&c->d_scal, (size_t)N * 4 * sizeof(double)));
  INIT_CU(cudaMalloc(&c->d_ek, c->total_cells * sizeof(double)));
  INIT_CU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  INIT_CU(cudaEventCreate(&c->ev0));
  INIT_CU(cudaEventCreate(&c->ev1));
  INIT_CU(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  {
    const char* g = getenv("RT_CNOP_GRAPHS");
    c->graphs = !(g && g[0] == '0');
    // fault injection for the TMA wait's timeout path: arm the barriers, issue
    // no copy, bound each wait by a few polls; every tile-kernel call then
    // fails with RT_ETIMEOUT and nothing is left in flight
    const char* f = getenv("RT_CNOP_TMA_WAIT_FAULT");
    const bool fault = f && f[0] == '1';
    c->run.tma_skip = fault ? 1 : 0;
    c->run.tma_polls = fault ? 16 : (1 << 18);
  }
  INIT_CU(c->esz == 8 ? rt::configure_kernels<double>() : rt::configure_kernels<float>());
  size_t freeb = 0, totb = 0;
  INIT_CU(cudaMemGetInfo(&freeb, &totb));
  c->mem_cap = c->opt.ckpt_hbm_cap_bytes > 0 ? c->opt.ckpt_hbm_cap_bytes : 0.6 * (double)freeb;
  bool need_base = false;
  for (int i = 0; i < N; ++i) need_base = need_base || c->prob[i].objective == RT_OBJ_EK_ANOMALY_L2;
  if (need_base) {
    rt_status s = ensure_fields(c, false);
    if (s == RT_OK) s = c->esz == 8 ? baseline<double>(c) : baseline<float>(c);
    if (s != RT_OK) return bail(s);
  }
  if (c->opt.stage_kernel == RT_STAGE_SWEEP || c->opt.stage_kernel == RT_STAGE_TILE ||
      c->opt.stage_kernel == RT_STAGE_TILE8 || c->opt.stage_kernel == RT_STAGE_TILE32) {
    c->stage_variant = c->opt.stage_kernel;
  } else if (c->opt.stage_kernel == RT_STAGE_AUTO) {
    rt_status s = ensure_fields(c, false);
    if (s == RT_OK) s = c->esz == 8 ? autotune_stage<double>(c) : autotune_stage<float>(c);
    if (s != RT_OK) return bail(s);
  } else {
    fail(c, RT_EINVAL, "stage_kernel");
    return bail(RT_EINVAL);
  }
  {
    rt_status s = ensure_fields(c, false);
    if (s == RT_OK) s = c->esz == 8 ? autotune_adjoint<double>(c) : autotune_adjoint<float>(c);
    if (s != RT_OK) return bail(s);
  }
#undef INIT_CU
  *out = c;
  return RT_OK;
}

void rt_destroy(rt_ctx* c) {
  if (!c) return;
  if (c->d_pinst && c->d_pinst != c->d_inst) cudaFree(c->d_pinst);
  if (c->d_tiles_h[0]) cudaFree(c->d_tiles_h[0]);
  if (c->d_tiles_h[2]) cudaFree(c->d_tiles_h[2]);
  if (c->d_tiles_a24) cudaFree(c->d_tiles_a24);
  void* ptrs[] = {c->d_inst, c->d_tiles, c->d_strips, c->d_base, c->d_base_f, c->d_ek0, c->d_ek, c->sA, c->sB, c->sU1, c->lA, c->lB,
                  c->l1, c->d_tab, c->run.dtrec, c->run.wrec, c->d_blast, c->d_coef, c->run.dtc, c->run.counter, c->run.t, c->run.nstep, c->run.wmin, c->run.status,
                  c->run.bad_cell, c->d_partials, c->d_sums, c->d_scal, c->d_v, c->d_g, c->d_w1, c->d_w2,
                  c->d_w3, c->d_w4, c->d_pairs, c->d_rows, c->d_rowsum, c->d_sample};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : c->pool) cudaFree(p);
  for (void* p : c->pool1) cudaFree(p);
  for (auto& kv : c->gcache) cudaGraphExecDestroy(kv.second.exec);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

const char* rt_last_error(const rt_ctx* c) { return c ? c->err.c_str() : "null context"; }

int rt_num_instances(const rt_ctx* c) { return c ? c->n_inst : 0; }
size_t rt_field_offset(const rt_ctx* c, int i) { return (c && i >= 0 && i < c->n_inst) ? c->v_off[i] : 0; }
size_t rt_field_size(const rt_ctx* c, int i) {
  if (!c || i < 0 || i >= c->n_inst) return 0;
  return (size_t)c->prob[i].perturb_ncomp * c->prob[i].nx * c->prob[i].ny;
}
size_t rt_field_total(const rt_ctx* c) { return c ? c->total_v : 0; }

rt_status rt_forward(rt_ctx* c, const double* v0, int flags, double* J_out, double* J_ke_out, rt_run_stats* st) {
  if (!c || !v0 || !J_out) return fail(c, RT_EINVAL, "null argument");
  Range range("rt_forward");
  c->err.clear();
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  reset_accounting(c);
  Timer tm(c);
  CHK(copy_in(c, v0, flags, c->d_v));
  int steps = 0;
  const rt_status s = c->esz == 8 ? forward_impl<double>(c, c->d_v, flags, J_out, J_ke_out, &steps)
                                  : forward_impl<float>(c, c->d_v, flags, J_out, J_ke_out, &steps);
  if (s != RT_OK) return failed_call(c, st, s);
  const float ms = tm.stop();
  collect_timing(c);
  fill_stats(c, st, ms, 0);
  return RT_OK;
}

rt_status rt_forward_series(rt_ctx* c, const double* v0, int flags, int every, int max_samples, double* t_out,
                            double* ke_out, double* hmix_out, int* n_out) {
  if (!c || !v0 || !t_out || !ke_out || !hmix_out || !n_out) return fail(c, RT_EINVAL, "null argument");
  if (every < 1 || max_samples < 1) return fail(c, RT_EINVAL, "every and max_samples must be >= 1");
  if (c->n_dev != c->n_inst) return fail(c, RT_EINVAL, "rt_forward_series is not available with y-slabs");
  c->err.clear();
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  reset_accounting(c);
  CHK(copy_in(c, v0, flags, c->d_v));
  std::vector<double> smp;
  CHK(c->esz == 8 ? series_impl<double>(c, c->d_v, flags, every, smp)
                  : series_impl<float>(c, c->d_v, flags, every, smp));
  const int N = c->n_inst;
  const size_t npts = smp.size() / (4 * (size_t)N);
  for (int i = 0; i < N; ++i) {
    int k = 0;
    double last = -1.0;
    for (size_t s = 0; s < npts && k < max_samples; ++s) {
      const double* q = smp.data() + (s * N + i) * 4;
      if (q[3] <= last) continue;  // no step since the previous sample
      last = q[3];
      t_out[(size_t)i * max_samples + k] = q[0];
      ke_out[(size_t)i * max_samples + k] = q[1];
      hmix_out[(size_t)i * max_samples + k] = q[2];
      ++k;
    }
    n_out[i] = k;
  }
  return RT_OK;
}


rt_status rt_spectrum_x(rt_ctx* c, const double* v, int flags, int inst, double* E_out, int* y_peak_out) {
  if (!c || !v || !E_out) return fail(c, RT_EINVAL, "null argument");
  if (inst < 0 || inst >= c->n_inst) return fail(c, RT_EINVAL, "instance %d out of range", inst);
  c->err.clear();
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  SpecWork w;
  CHK(spec_alloc(c, w));
  CHK(copy_in(c, v, flags, c->d_v));
  const rt_problem& P = c->prob[inst];
  const double* f = uy_plane(c, c->d_v, inst);
  const long long n = (long long)P.nx * P.ny;
  CU(rt::spec_real_to_complex(f, w.a, n, c->stream));
  CU(rt::spec_dft_x(w.a, w.b, P.nx, P.ny, -1.0, c->stream));
  CU(rt::spec_rms_peak(f, P.nx, P.ny, w.ints, c->stream));
  CU(rt::spec_select_x(w.b, P.nx, w.ints, 0, w.E, w.keep, w.ints + 1, c->stream));
  int yp = 0;
  CU(cudaMemcpyAsync(E_out, w.E, (P.nx / 2) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(&yp, w.ints, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (y_peak_out) *y_peak_out = yp;
  return RT_OK;
}

rt_status rt_spectrum_2d(rt_ctx* c, const double* v, int flags, int inst, double* E_out) {
  if (!c || !v || !E_out) return fail(c, RT_EINVAL, "null argument");
  if (inst < 0 || inst >= c->n_inst) return fail(c, RT_EINVAL, "instance %d out of range", inst);
  c->err.clear();
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  SpecWork w;
  CHK(spec_alloc(c, w));
  CHK(copy_in(c, v, flags, c->d_v));
  const rt_problem& P = c->prob[inst];
  const long long n = (long long)P.nx * P.ny;
  CU(rt::spec_real_to_complex(uy_plane(c, c->d_v, inst), w.a, n, c->stream));
  CU(rt::spec_dft_x(w.a, w.b, P.nx, P.ny, -1.0, c->stream));
  CU(rt::spec_dft_y(w.b, w.a, P.nx, P.ny, -1.0, c->stream));
  CU(rt::spec_power(w.a, w.E, n, c->stream));
  CU(rt::spec_select_pairs(w.E, P.nx, P.ny, 1.0, w.keep, w.ints + 1, w.dbl, c->stream));
  CU(rt::spec_scale_by(w.E, n, w.dbl, c->stream));
  CU(cudaMemcpyAsync(E_out, w.E, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_reconstruct(rt_ctx* c, const double* v, int flags, int kind, double param, const double* eps,
                         double* out, int* kept_out) {
  if (!c || !v || !eps || !out) return fail(c, RT_EINVAL, "null argument");
  if (kind == RT_RECON_X_MODES ? !(param >= 1.0) : kind == RT_RECON_2D_POWER ? !(param > 0.0 && param <= 1.0) : true)
    return fail(c, RT_EINVAL, "kind %d with parameter %g", kind, param);
  c->err.clear();
  CHK(ensure_fields(c, true));
  CHK(enter(c));
  SpecWork w;
  CHK(spec_alloc(c, w));
  CHK(copy_in(c, v, flags, c->d_v));
  double* r = c->d_w1;
  const int N = c->n_inst;
  for (int i = 0; i < N; ++i) {
    const rt_problem& P = c->prob[i];
    const long long n = (long long)P.nx * P.ny;
    const double* f = uy_plane(c, c->d_v, i);
    // mode set from u_y
    CU(rt::spec_real_to_complex(f, w.a, n, c->stream));
    CU(rt::spec_dft_x(w.a, w.b, P.nx, P.ny, -1.0, c->stream));
    if (kind == RT_RECON_X_MODES) {
      CU(rt::spec_rms_peak(f, P.nx, P.ny, w.ints, c->stream));
      const int count = (int)std::min(param, (double)(P.nx / 2));
      CU(rt::spec_select_x(w.b, P.nx, w.ints, count, w.E, w.keep, w.ints + 1, c->stream));
    } else {
      CU(rt::spec_dft_y(w.b, w.a, P.nx, P.ny, -1.0, c->stream));
      CU(rt::spec_power(w.a, w.E, n, c->stream));
      CU(rt::spec_select_pairs(w.E, P.nx, P.ny, param, w.keep, w.ints + 1, w.dbl, c->stream));
    }
    // that set applied to every perturbed component
    for (int k = 0; k < P.perturb_ncomp; ++k) {
      const size_t off = c->v_off[i] + (size_t)k * n;
      CU(rt::spec_real_to_complex(c->d_v + off, w.a, n, c->stream));
      CU(rt::spec_dft_x(w.a, w.b, P.nx, P.ny, -1.0, c->stream));
      if (kind == RT_RECON_X_MODES) {
        CU(rt::spec_mask(w.b, w.keep, P.nx, P.ny, 0, c->stream));
        CU(rt::spec_dft_x(w.b, w.a, P.nx, P.ny, 1.0, c->stream));
        CU(rt::spec_real_part(w.a, r + off, n, 1.0 / P.nx, c->stream));
      } else {
        CU(rt::spec_dft_y(w.b, w.a, P.nx, P.ny, -1.0, c->stream));
        CU(rt::spec_mask(w.a, w.keep, P.nx, P.ny, 1, c->stream));
        CU(rt::spec_dft_y(w.a, w.b, P.nx, P.ny, 1.0, c->stream));
        CU(rt::spec_dft_x(w.b, w.a, P.nx, P.ny, 1.0, c->stream));
        CU(rt::spec_real_part(w.a, r + off, n, 1.0 / ((double)P.nx * P.ny), c->stream));
      }
    }
    int kept = 0;
    CU(cudaMemcpyAsync(&kept, w.ints + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (kept_out) kept_out[i] = kept;
  }
  // rescale onto C = eps
  std::vector<double> C, sc(N);
  CHK(field_sums(c, 0, r, nullptr, C));
  for (int i = 0; i < N; ++i) {
    if (!(C[i] > 0.0) || !std::isfinite(C[i]))
      return fail(c, RT_EINVAL, "reconstruction of instance %d has C = %g", i, C[i]);
    sc[i] = std::sqrt(eps[i] / C[i]);
  }
  CHK(axpby(c, r, sc, r, nullptr, nullptr));
  CHK(copy_out(c, r, flags, out));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_gradient(rt_ctx* c, const double* v0, int flags, double* J_out, double* grad_out, rt_run_stats* st) {
  if (!c || !v0 || !J_out || !grad_out) return fail(c, RT_EINVAL, "null argument");
  Range range("rt_gradient");
  if (flags & RT_REPLAY_DT) return fail(c, RT_EINVAL, "rt_gradient runs its own step control (RT_REPLAY_DT is not accepted)");
  c->err.clear();
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  reset_accounting(c);
  Timer tm(c);
  CHK(copy_in(c, v0, flags, c->d_v));
  int segments = 0;
  const bool dtg = (flags & RT_GRAD_DT) != 0;
  const rt_status s = c->esz == 8 ? gradient_impl<double>(c, c->d_v, J_out, c->d_g, &segments, dtg)
                                  : gradient_impl<float>(c, c->d_v, J_out, c->d_g, &segments, dtg);
  if (s != RT_OK) return failed_call(c, st, s);
  CHK(copy_out(c, c->d_g, flags, grad_out));
  const float ms = tm.stop();
  collect_timing(c);
  fill_stats(c, st, ms, segments);
  return RT_OK;
}

rt_status rt_constraint(rt_ctx* c, const double* v, int flags, double* C_out) {
  if (!c || !v || !C_out) return fail(c, RT_EINVAL, "null argument");
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  CHK(copy_in(c, v, flags, c->d_v));
  std::vector<double> C;
  CHK(field_sums(c, 0, c->d_v, nullptr, C));
  std::copy(C.begin(), C.end(), C_out);
  return RT_OK;
}

rt_status rt_project(rt_ctx* c, double* v, int flags, const double* eps, int to_budget) {
  if (!c || !v || !eps) return fail(c, RT_EINVAL, "null argument");
  CHK(ensure_fields(c, false));
  CHK(enter(c));
  CHK(copy_in(c, v, flags, c->d_v));
  std::vector<double> C;
  CHK(field_sums(c, 0, c->d_v, nullptr, C));
  std::vector<double> sc(c->n_inst);
  for (int i = 0; i < c->n_inst; ++i) {
    if (!(C[i] > 0.0)) return fail(c, RT_EINVAL, "instance %d: C(v) = 0, cannot scale", i);
    sc[i] = (!to_budget && C[i] <= eps[i]) ? 1.0 : std::sqrt(eps[i] / C[i]);
  }
  CHK(axpby(c, c->d_v, sc, c->d_v, nullptr, nullptr));
  CHK(copy_out(c, c->d_v, flags, v));
  CU(cudaStreamSynchronize(c->stream));
  return RT_OK;
}

rt_status rt_get_state(rt_ctx* c, int inst, double* out) {
  if (!c || !out || inst < 0 || inst >= c->n_inst) return fail(c, RT_EINVAL, "bad argument");
  if (!c->have_run) return fail(c, RT_ESTATE, "no run yet");
  const rt_problem& P = c->prob[inst];
  const size_t n = (size_t)4 * P.nx * P.ny;
  const int s = c->h_nstep[inst];
  const void* slot = c->last_kind == 2 ? c->pool[s] : ((s & 1) ? c->sB : c->sA);
  // the owned rows of each of the problem's device instances (slabs), in order
  std::vector<char> raw(n * c->esz);
  long long row = 0;
  for (int d = c->dev_first[inst]; d < c->dev_first[inst] + c->dev_count[inst]; ++d) {
    const InstDev& I = c->h_inst[d];
    const size_t es = c->esz, own = (size_t)(I.own1 - I.own0) * I.nx;
    const char* src = static_cast<const char*>(slot) + ((size_t)4 * I.cell_off + (size_t)I.own0 * I.nx) * es;
    CU(cudaMemcpy2DAsync(raw.data() + (size_t)row * I.nx * es, (size_t)P.nx * P.ny * es, src,
                         (size_t)I.nx * I.ny * es, own * es, 4, cudaMemcpyDeviceToHost, c->stream));
    row += I.own1 - I.own0;
  }
  CU(cudaStreamSynchronize(c->stream));
  if (c->esz == 8) {
    std::memcpy(out, raw.data(), n * sizeof(double));
  } else {
    const float* f = reinterpret_cast<const float*>(raw.data());
    for (size_t k = 0; k < n; ++k) out[k] = f[k];
    // the FP32 state holds the deviation from the row's base state: add
    // rho0 to the density and p0/(gamma-1) to the energy
    const size_t cells = (size_t)P.nx * P.ny;
    const float* rb = c->h_base_f.data() + c->row_off[inst];
    const float* pb = rb + c->base_rows;
    const double gm1 = P.gamma - 1.0;
    for (int y = 0; y < P.ny; ++y)
      for (int x = 0; x < P.nx; ++x) {
        const size_t k = (size_t)y * P.nx + x;
        out[k] += (double)rb[y];
        out[3 * cells + k] += (double)pb[y] / gm1;
      }
  }
  return RT_OK;
}

rt_status rt_get_dt(rt_ctx* c, int inst, double* out, int max_n, int* n_out) {
  if (!c || inst < 0 || inst >= c->n_inst) return fail(c, RT_EINVAL, "bad argument");
  if (!c->have_run) return fail(c, RT_ESTATE, "no run yet");
  const int n = c->h_nstep[inst];
  if (n_out) *n_out = n;
  const int k = std::min(n, max_n);
  if (out && k > 0) {
    CU(cudaMemcpyAsync(out, c->run.dtrec + (size_t)inst * c->opt.max_steps, k * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
  }
  return RT_OK;
}

rt_status rt_set_kernel_timing(rt_ctx* c, int every) {
  if (!c || every < 0) return fail(c, RT_EINVAL, "bad argument");
  c->time_every = every;
  if (every > 0 && c->evpool.empty()) {
    c->evpool.resize(2 * 8192);
    for (auto& e : c->evpool) CU(cudaEventCreate(&e));
  }
  return RT_OK;
}

int rt_stage_kernel(const rt_ctx* c, double* tuned_ms) {
  if (!c) return 0;
  if (tuned_ms) {
    tuned_ms[0] = c->tune_ms[rt::STAGE_SWEEP];
    tuned_ms[1] = c->tune_ms[rt::STAGE_TILE];
  }
  return c->stage_variant;
}

rt_status rt_stage_tuning(const rt_ctx* c, double* ms) {
  if (!c || !ms) return RT_EINVAL;
  ms[0] = c->tune_ms[rt::STAGE_SWEEP];
  ms[1] = c->tune_ms[rt::STAGE_TILE8];
  ms[2] = c->tune_ms[rt::STAGE_TILE];
  ms[3] = c->tune_ms[rt::STAGE_TILE32];
  return RT_OK;
}

int rt_adjoint_rows(const rt_ctx* c, double* ms) {
  if (!c) return 0;
  if (ms) {
    ms[0] = c->adj_tune_ms[0];
    ms[1] = c->adj_tune_ms[1];
  }
  return c->adj_rows;
}

rt_status rt_kernel_times(rt_ctx* c, double* mean_ms, long long* samples, long long* launches) {
  if (!c) return RT_EINVAL;
  for (int k = 0; k < 3; ++k) {
    if (mean_ms) mean_ms[k] = c->kind_samples[k] ? c->kind_ms[k] / c->kind_samples[k] : 0.0;
    if (samples) samples[k] = c->kind_samples[k];
    if (launches) launches[k] = c->kind_launches[k];
  }
  return RT_OK;
}

rt_status cnop_solve(rt_ctx* c, const cnop_params* prm, double* v_inout, int flags, double* J_out,
                     cnop_result* res) {
  if (!c || !prm || !v_inout || !prm->eps) return fail(c, RT_EINVAL, "null argument");
  Range range("cnop_solve");
  if (prm->max_iter < 0) return fail(c, RT_EINVAL, "max_iter < 0");
  if (prm->lbfgs_memory < 0) return fail(c, RT_EINVAL, "lbfgs_memory < 0");
  c->err.clear();
  CHK(enter(c));
  Timer tm(c);
  rt_status s;
  if (prm->method == RT_CNOP_LBFGS || prm->method == RT_CNOP_SPG)
    s = c->esz == 8 ? cnop_run<double>(c, prm, v_inout, flags, J_out, res)
                    : cnop_run<float>(c, prm, v_inout, flags, J_out, res);
  else
    s = fail(c, RT_EINVAL, "unknown CNOP method %d", prm->method);
  const float ms = tm.stop();
  if (res) res->ms = ms;
  return s;
}

rt_status rt_tma_plan(const int* nx, const int* ny, int n, int elem_bytes, int* group_of, int* index_of) {
  if (!nx || !ny || n < 0 || (elem_bytes != 4 && elem_bytes != 8) || !group_of || !index_of) return RT_EINVAL;
  for (int i = 0; i < n; ++i) {
    group_of[i] = -1;
    index_of[i] = 0;
  }
  const std::vector<rt::TmaRun> runs =
      rt::tma_plan(nx, ny, n, (size_t)elem_bytes, kTmaMinNx, kTmaMinNy, rt::TMA_GROUPS);
  for (size_t g = 0; g < runs.size(); ++g)
    for (int k = 0; k < runs[g].count; ++k) {
      group_of[runs[g].first + k] = (int)g;
      index_of[runs[g].first + k] = k;
    }
  return RT_OK;
}

rt_status rt_revolve_plan(int steps, int slots, long long* recomputed, double* optimum) {
  if (steps < 0 || slots < 0) return RT_EINVAL;
  if (recomputed) *recomputed = rt::revolve_recomputed(steps, slots);
  if (optimum) *optimum = rt::revolve_optimum(steps, slots);
  return RT_OK;
}

}  // extern "C"
