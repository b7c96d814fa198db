// rwmi_api.cu -- host side of the C ABI declared in include/rwmi.h: context state, device
// memory, the per-step launch sequence (replayed from captured CUDA graphs), read-back and
// checkpointing. Every step of the method runs in the kernels of rwmi_fluid.cu, rwmi_lbm.cu,
// rwmi_walkers.cu and rwmi_dem.cu; this file only sequences them.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <map>
#include <string>
#include <vector>

#include "rwmi.h"
#include "rwmi_internal.cuh"

using namespace rwmi;

namespace {

constexpr int SERIES_ROWS = 65536;
constexpr int SERIES_COLS = 14;
constexpr int FORCE_ROWS = 4096;    // rows of the force series ring (1 + 6 P doubles each)
constexpr uint64_t CKPT_MAGIC = 0x31494d5752ULL;  // "RWMI1"
constexpr uint64_t CKPT_DEM_MAGIC = 0x314d4544ULL;  // "DEM1": the free-DEM section

// A captured run of steps is fixed by the buffer parities it starts from, its start time modulo
// the chunk (which steps sort and form moments) and its length.
struct GraphKey {
  int fcur, pcur;
  int64_t phase, len;
  bool operator<(const GraphKey& o) const {
    if (fcur != o.fcur) return fcur < o.fcur;
    if (pcur != o.pcur) return pcur < o.pcur;
    if (phase != o.phase) return phase < o.phase;
    return len < o.len;
  }
};
constexpr int64_t SEGMENT_MAX = 64;    // longest captured run of steps
constexpr size_t GRAPH_CACHE_MAX = 32;  // captured runs kept per context; beyond, runs are eager

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
};

}  // namespace

struct rwmi_ctx {
  // configuration
  int n[3];
  int64_t ncell;
  double tau, D;
  uint64_t seed;
  rwmi_config cfg;
  Geom g;
  int device = 0, nsm = 152;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;    // raster of t+1 beside the LBM of t
  cudaStream_t wst = nullptr;     // walkers of t beside the fluid of t+1
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr, fluid_ev = nullptr, walk_ev[2] = {nullptr, nullptr};
  bool stepped = false;
  std::string err;

  // device state
  void* f[2] = {nullptr, nullptr};
  CUtensorMap tmap[2];                // TMA maps of f[0], f[1] (TMA-staged LBM update)
  bool tma_ok = false;                // both encoded for the current q, storage and buffers
  float* u[2] = {nullptr, nullptr};   // (u, rho) per time parity: the LBM of t writes u[t & 1]
  uint16_t* solid[2] = {nullptr, nullptr};   // per time parity: raster of t+1 beside the LBM of t
  uint16_t* node[2] = {nullptr, nullptr};    // IBB node classes per time parity (0 fluid, 1 + particle)
  IbbLinks ibl;                              // IBB link list (allocated with coupling 1)
  int64_t* d_T = nullptr;
  unsigned long long* status = nullptr;
  double* acc[2] = {nullptr, nullptr};   // per time parity: forces [6P] + mass/momentum [4]
  double* macc = nullptr;                // moment accumulators [12]
  double* series = nullptr;              // [SERIES_ROWS][SERIES_COLS]
  double* mrow = nullptr;                // on-demand moments row [SERIES_COLS]
  double* fseries = nullptr;             // force series ring [FORCE_ROWS][1 + 6 P] (force_interval > 0)
  int fseries_p = 0;                     // particle count the ring was sized for
  // bricks per time parity (the walker masks are rewritten by every raster)
  uint64_t* wmask[2] = {nullptr, nullptr};
  uint32_t* bword[2] = {nullptr, nullptr};
  uint16_t* bcand[2] = {nullptr, nullptr};
  int32_t* rlist[2] = {nullptr, nullptr};
  PoseF* pose[2] = {nullptr, nullptr};
  StepParams* sp[2] = {nullptr, nullptr};
  float4* cworld[2] = {nullptr, nullptr};
  uint32_t nbrick = 0;
  // particles
  int P = 0, Nc = 0;
  ParticleDesc* desc = nullptr;
  float4* cbody = nullptr;
  float walk_margin = 1.0f;
  std::vector<float4> hbody;             // host copy of the body-frame control points
  std::vector<int> hcoff;                // [P + 1]
  // free DEM (rwmi_set_dem): one binary64 allocation for the state, parameters, contact memory
  // and slot forces (dem_layout), one byte allocation for the contact flags
  bool dem = false;
  rwmi_dem_config demcfg{};
  double* dem_d = nullptr;
  unsigned char* dem_b = nullptr;
  // walkers
  int64_t nw = 0;
  float4* pos[2] = {nullptr, nullptr};
  float4* x0[2] = {nullptr, nullptr};
  uint32_t* rank = nullptr;
  float4* wlist = nullptr;            // walkers flagged for the particle-resolution pass
  unsigned int* wlist_n = nullptr;
  uint32_t* counts = nullptr;
  uint32_t* offsets = nullptr;
  uint32_t* bsums = nullptr;
  // scratch for read-back conversions
  void* scratch = nullptr;
  size_t scratch_bytes = 0;

  // host mirrors
  int64_t t = 0;
  int64_t t_base = 0;   // value of the device counter d_T: t at the start of the current run
  bool walk_rec[2] = {false, false};   // walk_ev[p] recorded in the current run
  int fcur = 0, pcur = 0;
  int64_t binned_t = -1;
  int64_t series_rows = 0;
  int64_t fseries_rows = 0;
  int64_t launches = 0;
  unsigned long long status_seen[ST_COUNT] = {0};
  std::map<GraphKey, GraphEntry> graphs;
  // phase timing (rwmi_step_timed): events[phase] start/stop pairs when enabled
  bool timing = false;
  // Set by an allocation or CUDA failure: the device state may be half built, so every later
  // call but rwmi_last_error and rwmi_destroy is refused with RWMI_E_STATE.
  bool broken = false;
  cudaEvent_t ev[2 * RWMI_NPHASE] = {};
};

// Many contexts advanced together: one CUDA graph per chunk forks every context's steps onto
// its own stream (concurrent branches) and joins them on the batch's stream.
// Fused batch phases: each is one launch for every context of the batch.
enum FusedPhase {
  FP_CLEARB = 0, FP_POSE, FP_RASTER, FP_LBM, FP_WALK, FP_RESOLVE, FP_CLEARC, FP_HIST, FP_SCANR, FP_SCANT,
  FP_SCAND, FP_SCATTER, FP_MOM, FP_MOMFIN, FP_ADV, FP_COUNT
};
struct FusedGraph {
  cudaGraphExec_t exec = nullptr;
  void* args = nullptr;   // device argument records of every step of the chunk
  int64_t launches = 0;
};

struct rwmi_batch {
  std::vector<rwmi_ctx*> ctxs;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join;
  std::map<std::vector<int>, std::pair<cudaGraphExec_t, std::vector<int64_t>>> graphs;
  int64_t L = 2;
  std::string err;
  // fused execution (rwmi_batch_set_mode): one launch per phase for all contexts, each block
  // mapped to (context, block of that context's grid) through device block maps
  int mode = RWMI_BATCH_AUTO;
  bool fused = false;
  rwmi_batch_tiles tiles{128, 1, 8192, 64};
  cudaStream_t side = nullptr;           // raster of t+1 beside the LBM of t
  cudaStream_t wst = nullptr;            // walkers of t beside the fluid of t+1
  cudaEvent_t fork2 = nullptr, join2 = nullptr, fluid_ev = nullptr, walk_ev[2] = {nullptr, nullptr};
  BlockMap* maps = nullptr;              // device: the block maps of every phase, back to back
  size_t map_off[FP_COUNT] = {}, map_n[FP_COUNT] = {};
  std::map<std::vector<int>, FusedGraph> fgraphs;
  int64_t launches = 0;
};

namespace {

rwmi_status fail(rwmi_ctx* c, rwmi_status s, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (s == RWMI_E_OOM || s == RWMI_E_CUDA) c->broken = true;
  }
  return s;
}

// A C++ exception (host memory: std::bad_alloc, std::length_error) never crosses the C ABI: each
// entry point turns it into RWMI_E_OOM, which fences the context like a device allocation failure.
rwmi_status api_exception(rwmi_ctx* c, const char* fn, const std::exception& e) {
  return fail(c, RWMI_E_OOM, std::string(fn) + ": host allocation failed (" + e.what() + ")");
}

// A context fenced by an earlier failure refuses the call; its message stays the first failure's.
#define GUARD(c)                                \
  do {                                          \
    if ((c)->broken) return RWMI_E_STATE;       \
  } while (0)

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(c, e_ == cudaErrorMemoryAllocation ? RWMI_E_OOM : RWMI_E_CUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

// Device memory is stream-ordered on the context's stream: creating or destroying one context
// never synchronises the device, so other contexts' work keeps running meanwhile.
// Host-side fault injection (rwmi_inject_alloc_failure): the allocation whose process-wide
// index equals g_fail_at reports cudaErrorMemoryAllocation without reaching the allocator.
std::atomic<int64_t> g_alloc_count{0};
std::atomic<int64_t> g_fail_at{-1};

template <typename T>
cudaError_t dalloc(rwmi_ctx* c, T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  const int64_t k = g_alloc_count.fetch_add(1);
  int64_t at = k;
  if (g_fail_at.compare_exchange_strong(at, -1)) return cudaErrorMemoryAllocation;
  return cudaMallocAsync((void**)p, bytes, c->stream);
}

void dfree(rwmi_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

// Device scratch owned by one API call: freed, stream-ordered, on every return path.
template <typename T>
struct CallScratch {
  rwmi_ctx* c;
  T* p = nullptr;
  explicit CallScratch(rwmi_ctx* cc) : c(cc) {}
  CallScratch(const CallScratch&) = delete;
  CallScratch& operator=(const CallScratch&) = delete;
  ~CallScratch() { dfree(c, p); }
};

// Blocking copy ordered on the context's stream (never on the legacy default stream, which
// would wait for every other blocking stream of the process).
cudaError_t copy_now(rwmi_ctx* c, void* dst, const void* src, size_t bytes) {
  const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream);
  return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}

size_t storage_bytes(int storage) { return storage == 2 ? 2 : storage == 3 ? 8 : 4; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

rwmi_status copy_out(rwmi_ctx* c, void* dst, const void* src, size_t bytes) {
  const cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(dst, src, bytes, k, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RWMI_OK;
}

rwmi_status ensure_scratch(rwmi_ctx* c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return RWMI_OK;
  dfree(c, c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  CK(dalloc(c, &c->scratch, bytes));
  c->scratch_bytes = bytes;
  return RWMI_OK;
}

void drop_graphs(rwmi_ctx* c) {
  for (auto& kv : c->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
}

ParticleSet particle_set(const rwmi_ctx* c) {
  ParticleSet ps;
  ps.P = c->P;
  ps.Nc = c->Nc;
  ps.desc = c->desc;
  ps.cbody = c->cbody;
  ps.walk_margin = c->walk_margin;
  ps.dem = c->dem ? c->dem_d : nullptr;   // the state sits first in dem_d
  return ps;
}

// Bound radius of a particle about its body origin: with r = |x - o|, |x - x_i| >= r - |c_i|, so
// f <= sum k_i / (r - |c_i|)^2 once r > max |c_i|; beyond the unit crossing of that falling bound
// f stays below 1. Inflated a little, since it only has to be conservative.
float bound_radius(const float4* body, int c0, int c1) {
  double cmax = 0.0, ksum = 0.0;
  std::vector<double> cn;
  for (int i = c0; i < c1; ++i) {
    const double r = std::sqrt((double)body[i].x * body[i].x + (double)body[i].y * body[i].y +
                               (double)body[i].z * body[i].z);
    cn.push_back(r);
    cmax = std::max(cmax, r);
    ksum += body[i].w;
  }
  double lo = cmax, hi = cmax + std::sqrt(ksum) + 1e-9;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    double s = 0.0;
    for (size_t m = 0; m < cn.size(); ++m) s += (double)body[c0 + m].w / ((mid - cn[m]) * (mid - cn[m]));
    if (s > 1.0) lo = mid; else hi = mid;
  }
  return (float)(hi * (1.0 + 1e-6) + 1e-4);
}

// Free-DEM buffers of P particles: binary64 words (dem_args' views, the mass properties [10 P],
// then the binary32 reach cache, [P] float4 at an even word offset so that it is 16-byte
// aligned), then contact-flag bytes
size_t dem_posf_offset(size_t P) { return (104 * P + 15 * P * P + 1) & ~(size_t)1; }
size_t dem_doubles(size_t P) { return dem_posf_offset(P) + 2 * P; }
double* dem_props(const rwmi_ctx* c) { return c->dem_d + 94 * (size_t)c->P + 15 * (size_t)c->P * c->P; }
size_t dem_bytes(size_t P) { return P * P + 6 * P; }

// Views of a context's DEM buffers; the fluid force is that of time parity tp (step t's update)
DemArgs dem_args(const rwmi_ctx* c, int tp) {
  DemArgs a;
  const size_t P = (size_t)c->P, PP = P * P;
  a.P = c->P;
  for (int e = 0; e < 3; ++e) { a.n[e] = c->n[e]; a.wall[e] = c->g.wall[e]; a.g[e] = c->demcfg.gravity[e]; }
  a.desc = c->desc;
  a.cbody = c->cbody;
  double* b = c->dem_d;
  a.st = b; b += 13 * P;
  a.mass = b; b += P;
  a.Ib = b; b += 6 * P;
  a.Rs = b; b += P;
  a.zoom = b; b += P;
  a.xi = b; b += 3 * PP;
  a.xm = b; b += 3 * PP;
  a.xiw = b; b += 18 * P;
  a.xmw = b; b += 18 * P;
  a.pF = b; b += 3 * PP;
  a.pTi = b; b += 3 * PP;
  a.pTj = b; b += 3 * PP;
  a.wF = b; b += 18 * P;
  a.wT = b;
  a.posf = reinterpret_cast<float4*>(c->dem_d + dem_posf_offset(P));   // after the mass properties
  a.act = c->dem_b;
  a.actw = c->dem_b + PP;
  a.Fe = c->demcfg.hydro ? c->acc[tp] : nullptr;
  a.kn = c->demcfg.kn; a.etan = c->demcfg.eta_n; a.kt = c->demcfg.kt; a.etat = c->demcfg.eta_t;
  a.mus = c->demcfg.mu_s;
  a.dt = 1.0 / (double)c->demcfg.substeps;
  return a;
}

BrickSet brick_set(const rwmi_ctx* c, int par) {
  BrickSet b;
  b.wmask = c->wmask[par];
  b.bword = c->bword[par];
  b.bcand = c->bcand[par];
  b.rlist = c->rlist[par];
  b.pose = c->pose[par];
  b.posed = reinterpret_cast<PoseD*>(c->pose[par] + (c->P > 0 ? c->P : 1));   // 48 P bytes: aligned
  b.cworld = c->cworld[par];
  b.sp = c->sp[par];
  return b;
}

void update_margin(rwmi_ctx* c) {
  // regular walker step: |u| <= U_BOUND plus three normals of at most 4.5 each. A longer step
  // (|z_a| > 4.5 for some axis: ~2e-5 of steps) is flagged and resolved against all particles.
  c->walk_margin = U_BOUND + (float)std::sqrt(2.0 * c->D) * 4.5f * 1.7320508f + 0.01f;
  // IBB: a cell whose lattice neighbour (up to sqrt(3) away) is solid must lie in a flagged brick,
  // so that cells of other bricks skip the neighbour checks
  if (c->cfg.coupling == 1 && c->walk_margin < 1.75f) c->walk_margin = 1.75f;
}

// Brick lists, poses, body force and solid fraction of the current time; zeroes its accumulators.
rwmi_status build_current_frame(rwmi_ctx* c) {
  const int par = (int)(c->t & 1);
  if (c->cfg.coupling == 1 && c->P > 0) {   // IBB: node classes of t - 1 (the first step refills from them)
    const int pp = par ^ 1;
    launch_clear_u32(c->bword[pp], c->nbrick + BWORD_EXTRA, c->stream);
    launch_pose_bin(c->g, particle_set(c), brick_set(c, pp), c->d_T, -1, c->cfg.body_force,
                    c->cfg.force_period, 1, c->acc[pp], c->cfg.q, c->tau, c->stream);
    launch_nodes(c->cfg.q, c->cfg.storage, c->g, particle_set(c), brick_set(c, pp), c->node[pp], c->node[pp],
                 c->f[c->fcur], c->cfg.rho0, false, c->stream);
    c->launches += 3;
  }
  CK(cudaMemsetAsync(c->bword[par], 0, sizeof(uint32_t) * (c->nbrick + BWORD_EXTRA), c->stream));
  launch_pose_bin(c->g, particle_set(c), brick_set(c, par), c->d_T, 0, c->cfg.body_force,
                  c->cfg.force_period, 1, c->acc[par], c->cfg.q, c->tau, c->stream);
  c->launches++;
  if (c->P > 0) {
    launch_raster(c->g, particle_set(c), brick_set(c, par), c->solid[par], c->status, c->nsm, c->stream);
    c->launches++;
  }
  CK(cudaGetLastError());
  return RWMI_OK;
}

rwmi_status reset_fluid(rwmi_ctx* c) {
  const double u0[3] = {c->cfg.init_velocity[0], c->cfg.init_velocity[1], c->cfg.init_velocity[2]};
  launch_init_populations(c->cfg.q, c->cfg.storage, c->g, c->f[c->fcur], c->cfg.rho0, u0,
                          c->u[(c->t + 1) & 1], c->stream);
  c->launches++;
  CK(cudaGetLastError());
  return RWMI_OK;
}

// The force series ring (force_interval > 0 with particles), sized for the current particle count.
rwmi_status ensure_force_series(rwmi_ctx* c) {
  if (c->cfg.force_interval <= 0 || c->P == 0) return RWMI_OK;
  if (c->fseries && c->fseries_p == c->P) return RWMI_OK;
  dfree(c, c->fseries);
  c->fseries = nullptr;
  CK(dalloc(c, &c->fseries, sizeof(double) * (size_t)FORCE_ROWS * (1 + 6 * (size_t)c->P)));
  c->fseries_p = c->P;
  c->fseries_rows = 0;
  return RWMI_OK;
}

// Tensor maps of the population buffers for the TMA-staged update, where it applies.
void update_tma(rwmi_ctx* c) {
  c->tma_ok = c->f[0] && c->f[1] && lbm_tma_supported(c->cfg.q, c->cfg.storage, c->g) &&
              lbm_tma_encode(c->cfg.q, c->cfg.storage, c->g, c->f[0], &c->tmap[0]) &&
              lbm_tma_encode(c->cfg.q, c->cfg.storage, c->g, c->f[1], &c->tmap[1]);
}

rwmi_status alloc_fluid(rwmi_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    dfree(c, c->f[k]);
    c->f[k] = nullptr;
  }
  const size_t pop = (size_t)c->cfg.q * c->g.ncell_pad * storage_bytes(c->cfg.storage);
  for (int k = 0; k < 2; ++k) CK(dalloc(c, &c->f[k], pop));
  update_tma(c);
  return RWMI_OK;
}

rwmi_status alloc_particles(rwmi_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    dfree(c, c->pose[k]);
    dfree(c, c->cworld[k]);
    dfree(c, c->acc[k]);
    c->pose[k] = nullptr;
    c->cworld[k] = nullptr;
    c->acc[k] = nullptr;
    CK(dalloc(c, &c->pose[k], (sizeof(PoseF) + sizeof(PoseD)) * (size_t)(c->P > 0 ? c->P : 1)));
    CK(dalloc(c, &c->cworld[k], sizeof(float4) * (size_t)(c->Nc > 0 ? c->Nc : 1)));
    CK(dalloc(c, &c->acc[k], sizeof(double) * (size_t)(6 * c->P + 4 * RED_SLOTS)));
    CK(cudaMemsetAsync(c->acc[k], 0, sizeof(double) * (size_t)(6 * c->P + 4 * RED_SLOTS), c->stream));
  }
  return RWMI_OK;
}

rwmi_status alloc_walkers(rwmi_ctx* c, int64_t n) {
  for (int k = 0; k < 2; ++k) {
    dfree(c, c->pos[k]);
    dfree(c, c->x0[k]);
    c->pos[k] = nullptr;
    c->x0[k] = nullptr;
  }
  dfree(c, c->rank);
  dfree(c, c->wlist);
  c->rank = nullptr;
  c->wlist = nullptr;
  c->nw = 0;
  for (int k = 0; k < 2; ++k) {
    CK(dalloc(c, &c->pos[k], sizeof(float4) * (size_t)n));
    CK(dalloc(c, &c->x0[k], sizeof(float4) * (size_t)n));
  }
  CK(dalloc(c, &c->rank, sizeof(uint32_t) * (size_t)n));
  CK(dalloc(c, &c->wlist, 2 * sizeof(float4) * (size_t)(WLIST_STRIPES * wlist_stripe_cap(n))));
  c->nw = n;
  c->pcur = 0;
  c->binned_t = -1;
  drop_graphs(c);
  // the flagged-walker list counters of both parities start at zero for new walkers
  CK(cudaMemsetAsync(c->wlist_n, 0, sizeof(unsigned int) * 2 * WLIST_STRIPES, c->stream));
  return RWMI_OK;
}

// Counting sort of the walkers by cell; the histogram is the concentration of Eq. 16.
void enqueue_sort(rwmi_ctx* c, cudaStream_t st) {
  launch_clear_u32(c->counts, (uint32_t)c->ncell, st);
  launch_histogram(c->g, c->pos[c->pcur], c->nw, c->counts, c->rank, st);
  launch_scan(c->counts, c->offsets, c->bsums, (uint32_t)c->ncell, st);
  launch_scatter(c->g, c->pos[c->pcur], c->x0[c->pcur], c->nw, c->offsets, c->rank,
                 c->pos[c->pcur ^ 1], c->x0[c->pcur ^ 1], st);
  c->launches += 6;
  c->pcur ^= 1;
}

void phase_begin(rwmi_ctx* c, int ph) {
  if (c->timing) cudaEventRecord(c->ev[2 * ph], c->stream);
}
void phase_end(rwmi_ctx* c, int ph) {
  if (c->timing) cudaEventRecord(c->ev[2 * ph + 1], c->stream);
}

// Are the forces of the step that completes step count `done` recorded in the force series?
bool force_recorded(const rwmi_ctx* c, int64_t done) {
  return c->cfg.force_interval > 0 && c->P > 0 && c->fseries && done % c->cfg.force_interval == 0;
}

// Storages with the fused update-and-reduce pass (launch_lbm's `fused`).
static bool fused_storage(int storage) { return storage == RWMI_STORE_FP32_SHIFT || storage == RWMI_STORE_FP64_SHIFT; }

// One timestep t -> t+1 of a run of steps (host mirrors advance as the launches are queued).
// Buffers are per time parity where two steps' kernels may overlap: the solid fraction of t is
// solid[t & 1] (rasterised during step t-1, or at set-up), the LBM of t writes u[t & 1], the
// raster of t+1 writes solid/wmask[(t+1) & 1], and bricks of t+1 are bricks[(t+1) & 1].
// Schedules (cfg.overlap; rwmi_step_timed always takes 0 so that each phase is timed alone):
//   0  one stream: LBM(t), poses(t+1), raster(t+1), walkers(t), sort/moments.
//   1  poses(t+1) first; raster(t+1) on the side stream while LBM(t) runs on the main one (the
//      raster is ALU-bound, the LBM HBM-bound); join; walkers on the main stream.
//   2  as 1, and the walkers (with sort and moments) run on their own stream, one step behind
//      the fluid: walkers(t) overlap LBM(t+1) and raster(t+2). Step t+2's fluid work waits for
//      walkers(t), the last reader of the parity it overwrites.
// Kernels take their time as d_T + offset (d_T = t at the start of the run), so concurrent
// steps never race on a counter; segment_end advances d_T once per run. `reduce`: also form the
// FP64 mass/momentum sums of this step.
void enqueue_step(rwmi_ctx* c, bool reduce) {
  const bool rec_f = force_recorded(c, c->t + 1);   // this step's forces go to the force series
  reduce = reduce || rec_f;
  const int tp = (int)(c->t & 1), tn = tp ^ 1;
  const int toff = (int)(c->t - c->t_base);
  const ParticleSet ps = particle_set(c);
  const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
  const int level = c->timing ? 0 : c->cfg.overlap;
  const bool fork_raster = level >= 1 && c->P > 0;
  cudaStream_t ws = level >= 2 ? c->wst : c->stream;
  if (ws != c->stream && c->walk_rec[tp]) cudaStreamWaitEvent(c->stream, c->walk_ev[tp], 0);
  const bool dem = c->dem && c->P > 0;
  auto pose = [&]() {   // particles, bricks and body force of t+1
    phase_begin(c, RWMI_PHASE_POSE);
    if (dem) {   // free DEM from t to t+1 with the fluid force of the LBM update of t
      c->launches += launch_dem(dem_args(c, tp), c->demcfg.substeps, c->stream);
    }
    launch_clear_u32(c->bword[tn], c->nbrick + BWORD_EXTRA, c->stream);
    c->launches++;
    launch_pose_bin(c->g, ps, brick_set(c, tn), c->d_T, toff + 1, c->cfg.body_force, c->cfg.force_period, 1,
                    c->acc[tn], c->cfg.q, c->tau, c->stream);
    c->launches++;
    phase_end(c, RWMI_PHASE_POSE);
  };
  const bool ibb = c->cfg.coupling == 1 && c->P > 0;
  auto lbm = [&]() {    // LBM at t
    phase_begin(c, RWMI_PHASE_LBM);
    IbbArgs ia;
    if (ibb) {   // node classes of t, refilling of nodes uncovered since t - 1
      launch_nodes(c->cfg.q, c->cfg.storage, c->g, ps, brick_set(c, tp), c->node[tn], c->node[tp],
                   c->f[c->fcur], c->cfg.rho0, true, c->stream);
      c->launches++;
      ia.nodes = c->node[tp];
      ia.uprev = reinterpret_cast<const float4*>(c->u[tn]);
      ia.desc = c->desc;
      launch_ibb_links(c->cfg.q, c->cfg.storage, c->g, brick_set(c, tp), c->node[tp], c->ibl, tp, c->desc,
                       c->f[c->fcur], c->u[tn], c->cfg.rho0, c->status, c->nsm, c->stream);
      c->launches += 2;
      ia.base = c->ibl.base;
      ia.word = c->ibl.word;
      ia.q = c->ibl.q;
      ia.g = c->ibl.g;
      ia.cap = c->ibl.cap;
    }
    // the partially saturated update through TMA-staged rows where it applies (same results).
    // Reduction steps run the update and the sums in one fused pass (binary32-shifted and
    // binary64 storage): its update arithmetic is bit-identical to the plain update's, which a
    // GPU test checks for every instantiation, so the trajectory does not depend on which steps
    // are reduced; the other storages add the reduce-only pass.
    const bool staged = !ibb && !dem && c->tma_ok && c->cfg.lbm_staging;
    if (staged)
      launch_lbm_tma(c->cfg.q, c->cfg.storage, c->tmap[c->fcur], c->g, c->f[c->fcur], c->f[c->fcur ^ 1], c->u[tp],
                     c->solid[tp], brick_set(c, tp), c->tau, c->cfg.rho0, c->status, c->nsm, c->stream);
    if (!staged || reduce)
      launch_lbm(c->cfg.q, c->cfg.storage, reduce, c->g, c->f[c->fcur], c->f[c->fcur ^ 1], c->u[tp], c->solid[tp],
                 brick_set(c, tp), c->tau, c->cfg.rho0, c->acc[tp] + 6 * c->P, c->acc[tp],
                 c->status, c->stream, c->cfg.lbm_block, ibb ? &ia : nullptr, dem || (reduce && !staged), !staged);
    // staged: the TMA update, plus the reduce-only pass on reduction steps; otherwise one pass,
    // or the update and the reduce-only pass for storages without the fused one (free DEM runs
    // only with storages that have it)
    if (staged) c->launches += reduce ? 2 : 1;
    else c->launches += (reduce && !fused_storage(c->cfg.storage)) ? 2 : 1;
    if (rec_f) {
      launch_force_row(c->acc[tp], c->P, c->fseries, c->cfg.force_interval, FORCE_ROWS, c->d_T, toff + 1,
                       c->stream);
      c->launches++;
      c->fseries_rows++;
    }
    phase_end(c, RWMI_PHASE_LBM);
    c->fcur ^= 1;
  };
  if (dem) {   // the particles of t+1 follow from the fluid force of t: raster after the LBM
    lbm();
    pose();
    phase_begin(c, RWMI_PHASE_RASTER);
    launch_raster(c->g, ps, brick_set(c, tn), c->solid[tn], c->status, c->nsm, c->stream, !ibb);
    c->launches++;
    phase_end(c, RWMI_PHASE_RASTER);
  } else if (fork_raster) {
    pose();
    cudaEventRecord(c->fork_ev, c->stream);
    cudaStreamWaitEvent(c->side, c->fork_ev, 0);
    launch_raster(c->g, ps, brick_set(c, tn), c->solid[tn], c->status, c->nsm, c->side, !ibb);
    c->launches++;
    cudaEventRecord(c->join_ev, c->side);
    lbm();
    cudaStreamWaitEvent(c->stream, c->join_ev, 0);
  } else {
    lbm();
    pose();
    phase_begin(c, RWMI_PHASE_RASTER);
    if (c->P > 0) {
      launch_raster(c->g, ps, brick_set(c, tn), c->solid[tn], c->status, c->nsm, c->stream, !ibb);
      c->launches++;
    }
    phase_end(c, RWMI_PHASE_RASTER);
  }
  // walkers t -> t+1: u of t, particles of t+1
  if (ws != c->stream) {
    cudaEventRecord(c->fluid_ev, c->stream);
    cudaStreamWaitEvent(ws, c->fluid_ev, 0);
  }
  phase_begin(c, RWMI_PHASE_WALKERS);
  if (c->nw > 0) {
    launch_walkers(c->g, ps, brick_set(c, tn), c->pos[c->pcur], c->nw, c->u[tp], c->d_T, toff, tp, (float)c->D,
                   k0, k1, c->status, c->wlist, c->wlist_n, c->nsm, ws);
    c->launches += 2;
  }
  phase_end(c, RWMI_PHASE_WALKERS);
  c->t += 1;
  phase_begin(c, RWMI_PHASE_SORT);
  if (c->nw > 0 && c->cfg.sort_interval > 0 && c->t % c->cfg.sort_interval == 0) {
    enqueue_sort(c, ws);
    c->binned_t = c->t;
  }
  phase_end(c, RWMI_PHASE_SORT);
  phase_begin(c, RWMI_PHASE_MOMENTS);
  if (c->cfg.moment_interval > 0 && c->t % c->cfg.moment_interval == 0) {
    launch_moments(c->pos[c->pcur], c->x0[c->pcur], c->nw, c->macc, c->series, c->cfg.moment_interval,
                   SERIES_ROWS, c->d_T, toff + 1, ws);
    c->launches += c->nw > 0 ? 2 : 1;
    c->series_rows++;
  }
  phase_end(c, RWMI_PHASE_MOMENTS);
  if (ws != c->stream) {
    cudaEventRecord(c->walk_ev[tp], ws);
    c->walk_rec[tp] = true;
  }
}

// Closes a run of steps: the main stream joins the walker stream, and one launch advances the
// device counter d_T by the run's length (no kernel of the run is still reading it).
void segment_end(rwmi_ctx* c) {
  if (c->walk_rec[0] || c->walk_rec[1]) {
    cudaStreamWaitEvent(c->stream, c->walk_ev[(c->t - 1) & 1], 0);
    c->walk_rec[0] = c->walk_rec[1] = false;
  }
  if (c->t > c->t_base) {
    launch_advance(c->d_T, c->t - c->t_base, c->stream);
    c->launches++;
    c->t_base = c->t;
  }
}

// Host mirrors of a replayed chunk of L steps (what enqueue_step does while capturing).
void advance_mirrors(rwmi_ctx* c, int64_t L) {
  for (int64_t s = 0; s < L; ++s) {
    c->fcur ^= 1;
    c->t += 1;
    if (c->nw > 0 && c->cfg.sort_interval > 0 && c->t % c->cfg.sort_interval == 0) {
      c->pcur ^= 1;
      c->binned_t = c->t;
    }
    if (c->cfg.moment_interval > 0 && c->t % c->cfg.moment_interval == 0) c->series_rows++;
    if (force_recorded(c, c->t)) c->fseries_rows++;
  }
  c->t_base = c->t;
}

int64_t chunk_length(const rwmi_ctx* c) {
  auto gcd = [](int64_t a, int64_t b) { while (b) { int64_t t = a % b; a = b; b = t; } return a; };
  int64_t L = 2;
  for (int64_t v : {(int64_t)c->cfg.sort_interval, (int64_t)c->cfg.moment_interval, (int64_t)c->cfg.force_interval})
    if (v > 0) L = L / gcd(L, v) * v;
  return L;
}

}  // namespace

// ============================================================================================
// Exported C ABI
// ============================================================================================
extern "C" {

RWMI_API void rwmi_config_defaults(rwmi_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->q = 19;
  cfg->storage = RWMI_STORE_FP32_SHIFT;
  cfg->wall_mask = 0;
  cfg->force_period = 0.0;
  cfg->rho0 = 1.0;
  cfg->sort_interval = 16;
  cfg->moment_interval = 0;
  cfg->use_graphs = 1;
  cfg->lbm_block = 128;
  cfg->overlap = 2;
  cfg->lbm_staging = 0;
}

RWMI_API rwmi_status rwmi_create(rwmi_ctx** out, const int32_t dims[3], double tau, double D,
                                 uint64_t seed) try {
  if (!out || !dims) return RWMI_E_INVALID;
  *out = nullptr;
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1 || dims[a] > (1 << 20)) return RWMI_E_INVALID;
    ncell *= dims[a];
  }
  if (ncell > 0x7fffffffLL || !(tau > 0.5) || !std::isfinite(tau) || !(D >= 0.0) || !std::isfinite(D))
    return RWMI_E_INVALID;
  rwmi_ctx* c = new rwmi_ctx();
  for (int a = 0; a < 3; ++a) c->n[a] = dims[a];
  c->ncell = ncell;
  c->tau = tau;
  c->D = D;
  c->seed = seed;
  rwmi_config_defaults(&c->cfg);
  Geom& g = c->g;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = dims[a];
    g.nb[a] = (dims[a] + BRICK - 1) / BRICK;
    g.wall[a] = 0;
  }
  g.nxy = (uint32_t)dims[0] * (uint32_t)dims[1];
  g.ncell = (uint32_t)ncell;
  // plane stride: a multiple of 64 values (128-byte aligned planes at every storage width),
  // with at least one spare slot past the last cell, where the LBM kernel's tail lanes store
  g.ncell_pad = (uint32_t)((ncell + 64) / 64 * 64);
  for (int a = 0; a < 3; ++a) g.inv_n[a] = 1.0f / (float)dims[a];
  make_divisor((uint32_t)dims[0], g.mx, g.sx);
  make_divisor(g.nxy, g.mxy, g.sxy);
  c->nbrick = (uint32_t)g.nb[0] * g.nb[1] * g.nb[2];
  update_margin(c);
  rwmi_status st = RWMI_OK;
  try {
    st = [&]() -> rwmi_status {
      CK(cudaGetDevice(&c->device));
      CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
      CK(cudaStreamCreate(&c->stream));
      c->own_stream = true;
      rwmi_status s = alloc_fluid(c);
      if (s != RWMI_OK) return s;
      for (int k = 0; k < 2; ++k) CK(dalloc(c, &c->u[k], sizeof(float4) * (size_t)g.ncell_pad));
      for (int k = 0; k < 2; ++k) CK(dalloc(c, &c->solid[k], sizeof(uint16_t) * (size_t)ncell));
      for (int k = 0; k < 2; ++k) CK(dalloc(c, &c->node[k], sizeof(uint16_t) * (size_t)ncell));
      CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      CK(cudaStreamCreateWithFlags(&c->wst, cudaStreamNonBlocking));
      for (cudaEvent_t* e : {&c->fork_ev, &c->join_ev, &c->fluid_ev, &c->walk_ev[0], &c->walk_ev[1]})
        CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
      CK(dalloc(c, &c->d_T, sizeof(int64_t)));
      CK(dalloc(c, &c->wlist_n, sizeof(unsigned int) * 2 * WLIST_STRIPES));
      CK(cudaMemsetAsync(c->wlist_n, 0, sizeof(unsigned int) * 2 * WLIST_STRIPES, c->stream));
      CK(dalloc(c, &c->status, sizeof(unsigned long long) * ST_COUNT));
      CK(dalloc(c, &c->macc, sizeof(double) * 12));
      CK(dalloc(c, &c->series, sizeof(double) * (size_t)SERIES_ROWS * SERIES_COLS));
      CK(dalloc(c, &c->mrow, sizeof(double) * SERIES_COLS));
      CK(dalloc(c, &c->counts, sizeof(uint32_t) * (size_t)ncell));
      for (int k = 0; k < 2; ++k) CK(dalloc(c, &c->wmask[k], sizeof(uint64_t) * c->nbrick));
      CK(dalloc(c, &c->offsets, sizeof(uint32_t) * (size_t)ncell));
      CK(dalloc(c, &c->bsums, sizeof(uint32_t) * scan_block_sums_size((uint32_t)ncell)));
      for (int k = 0; k < 2; ++k) {
        CK(dalloc(c, &c->bword[k], sizeof(uint32_t) * (c->nbrick + BWORD_EXTRA)));
        CK(dalloc(c, &c->bcand[k], sizeof(uint16_t) * (size_t)c->nbrick * MAXC));
        CK(dalloc(c, &c->rlist[k], sizeof(int32_t) * c->nbrick));
        CK(dalloc(c, &c->sp[k], sizeof(StepParams) + sizeof(GuoPairs)));   // GuoPairs follows
        CK(cudaMemsetAsync(c->sp[k], 0, sizeof(StepParams) + sizeof(GuoPairs), c->stream));
      }
      CK(dalloc(c, &c->desc, sizeof(ParticleDesc)));
      CK(dalloc(c, &c->cbody, sizeof(float4)));
      s = alloc_particles(c);
      if (s != RWMI_OK) return s;
      CK(cudaMemsetAsync(c->d_T, 0, sizeof(int64_t), c->stream));
      CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned long long) * ST_COUNT, c->stream));
      CK(cudaMemsetAsync(c->macc, 0, sizeof(double) * 12, c->stream));
      for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(c->solid[k], 0, sizeof(uint16_t) * (size_t)ncell, c->stream));
      for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(c->node[k], 0, sizeof(uint16_t) * (size_t)ncell, c->stream));
      s = reset_fluid(c);
      if (s != RWMI_OK) return s;
      s = build_current_frame(c);
      if (s != RWMI_OK) return s;
      CK(cudaStreamSynchronize(c->stream));
      return RWMI_OK;
    }();
  } catch (const std::exception& e_) {
    st = api_exception(c, "rwmi_create", e_);
  }
  if (st != RWMI_OK) {
    const std::string msg = c->err;
    rwmi_destroy(c);
    std::fprintf(stderr, "rwmi_create: %s\n", msg.c_str());
    return st;
  }
  *out = c;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return RWMI_E_OOM;
}

RWMI_API rwmi_status rwmi_configure(rwmi_ctx* c, const rwmi_config* cfg) try {
  if (!c || !cfg) return RWMI_E_INVALID;
  GUARD(c);
  if (c->stepped) return fail(c, RWMI_E_STATE, "rwmi_configure: only before the first step");
  if ((cfg->q != 15 && cfg->q != 19) || cfg->storage < 0 || cfg->storage > 3 || cfg->wall_mask > 7 ||
      !(cfg->rho0 > 0.0) || cfg->sort_interval < 0 || cfg->moment_interval < 0 ||
      !(cfg->force_period >= 0.0) ||
      !(cfg->lbm_block == 0 || cfg->lbm_block == 64 || cfg->lbm_block == 128 || cfg->lbm_block == 256) ||
      cfg->overlap < 0 || cfg->overlap > 2 || cfg->coupling < 0 || cfg->coupling > 1 ||
      cfg->lbm_staging < 0 || cfg->lbm_staging > 1 || cfg->force_interval < 0 ||
      (cfg->coupling == 1 && cfg->storage != RWMI_STORE_FP32_SHIFT && cfg->storage != RWMI_STORE_FP64_SHIFT))
    return fail(c, RWMI_E_INVALID, "rwmi_configure: bad q, storage, wall_mask, rho0 or interval");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(cfg->body_force[a]) || !std::isfinite(cfg->init_velocity[a]))
      return fail(c, RWMI_E_INVALID, "rwmi_configure: non-finite force or velocity");
  if (c->dem && cfg->storage != RWMI_STORE_FP32_SHIFT && cfg->storage != RWMI_STORE_FP64_SHIFT)
    return fail(c, RWMI_E_INVALID, "rwmi_configure: the free DEM needs storage 1 or 3");
  const bool realloc_f = cfg->q != c->cfg.q || cfg->storage != c->cfg.storage;
  c->cfg = *cfg;
  update_margin(c);
  for (int a = 0; a < 3; ++a) c->g.wall[a] = (cfg->wall_mask >> a) & 1;
  drop_graphs(c);
  if (realloc_f) {
    rwmi_status s = alloc_fluid(c);
    if (s != RWMI_OK) return s;
  }
  c->fcur = 0;
  if (cfg->coupling == 1 && !c->ibl.base) {
    // IBB link list: half a link per cell (2^20 at least); overflow slots of 18 links (Q - 1 at
    // most) for a sixteenth of the cells (2^16 at least). RWMI_IBB_LINK_CAP, if set, shrinks the
    // list (tests use it to run the overflow slots).
    int64_t cap = std::max<int64_t>(c->ncell / 2, 1 << 20);
    if (const char* e = std::getenv("RWMI_IBB_LINK_CAP")) cap = std::max<int64_t>(1, std::atoll(e));
    c->ibl.cap = (int)std::min<int64_t>(cap, 0x3fffffff);
    c->ibl.ocap = (int)std::min<int64_t>(std::max<int64_t>(c->ncell / 16, 1 << 16), 0x3fffffff / 18);
    const size_t nlq = (size_t)c->ibl.cap + (size_t)c->ibl.ocap * 18;
    CK(dalloc(c, &c->ibl.base, sizeof(int32_t) * (size_t)c->ncell));
    CK(dalloc(c, &c->ibl.word, sizeof(uint32_t) * (size_t)c->ncell));
    CK(dalloc(c, &c->ibl.cell, sizeof(uint32_t) * (size_t)c->ibl.cap));
    CK(dalloc(c, &c->ibl.meta, sizeof(uint32_t) * (size_t)c->ibl.cap));
    CK(dalloc(c, &c->ibl.q, sizeof(float) * nlq));
    CK(dalloc(c, &c->ibl.g, sizeof(double) * nlq));
    CK(dalloc(c, &c->ibl.ocell, sizeof(int32_t) * (size_t)c->ibl.ocap));
    CK(dalloc(c, &c->ibl.count, sizeof(unsigned int) * 4));
  }
  if (c->ibl.count) CK(cudaMemsetAsync(c->ibl.count, 0, sizeof(unsigned int) * 4, c->stream));
  rwmi_status s = ensure_force_series(c);
  if (s != RWMI_OK) return s;
  s = reset_fluid(c);
  if (s != RWMI_OK) return s;
  s = build_current_frame(c);
  if (s != RWMI_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_configure", e_);
}

RWMI_API rwmi_status rwmi_set_stream(rwmi_ctx* c, void* stream) try {
  if (!c) return RWMI_E_INVALID;
  GUARD(c);
  CK(cudaStreamSynchronize(c->stream));
  if (stream == nullptr) return RWMI_OK;   // keep the context's own (blocking) stream
  if (c->own_stream) cudaStreamDestroy(c->stream);
  c->own_stream = false;
  c->stream = (cudaStream_t)stream;
  drop_graphs(c);
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_set_stream", e_);
}

RWMI_API rwmi_status rwmi_set_metaballs(rwmi_ctx* c, int32_t P, const int32_t* coff, const float* cb,
                                        const float* k, const double* origin, const double* amplitude,
                                        const double* period, const double* phase, const double* omega) try {
  if (!c) return RWMI_E_INVALID;
  GUARD(c);
  if (c->stepped) return fail(c, RWMI_E_STATE, "rwmi_set_metaballs: only before the first step");
  if (P < 0 || P > MAX_PARTICLES) return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: 0 <= P <= 511");
  if (P > 0 && (!coff || !cb || !k || !origin || !amplitude || !period || !phase))
    return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: null array");
  const int Nc = P > 0 ? coff[P] : 0;
  if (Nc < 0 || Nc > MAX_CENTERS || (P > 0 && coff[0] != 0))
    return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: bad center offsets");
  std::vector<ParticleDesc> desc((size_t)(P > 0 ? P : 1));
  std::vector<float4> body((size_t)(Nc > 0 ? Nc : 1));
  for (int p = 0; p < P; ++p) {
    if (coff[p + 1] <= coff[p]) return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: empty particle");
    ParticleDesc& d = desc[p];
    for (int a = 0; a < 3; ++a) {
      d.org[a] = origin[3 * p + a];
      d.amp[a] = amplitude[3 * p + a];
      d.omega[a] = omega ? omega[3 * p + a] : 0.0;
      if (!std::isfinite(d.org[a]) || !std::isfinite(d.amp[a]) || !std::isfinite(d.omega[a]))
        return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: non-finite trajectory");
    }
    d.period = period[p];
    d.phase = phase[p];
    if (!(d.period >= 0.0) || !std::isfinite(d.phase))
      return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: bad period or phase");
    d.c0 = coff[p];
    d.c1 = coff[p + 1];
    for (int i = d.c0; i < d.c1; ++i) {
      if (!(k[i] > 0.0f) || !std::isfinite(cb[3 * i]) || !std::isfinite(cb[3 * i + 1]) || !std::isfinite(cb[3 * i + 2]))
        return fail(c, RWMI_E_INVALID, "rwmi_set_metaballs: bad control point");
      body[i] = make_float4(cb[3 * i], cb[3 * i + 1], cb[3 * i + 2], k[i]);
    }
    d.rb = bound_radius(body.data(), d.c0, d.c1);
  }
  dfree(c, c->desc);
  dfree(c, c->cbody);
  c->desc = nullptr;
  c->cbody = nullptr;
  dfree(c, c->dem_d);
  dfree(c, c->dem_b);
  c->dem_d = nullptr;
  c->dem_b = nullptr;
  c->dem = false;   // new particles follow their prescribed trajectories until rwmi_set_dem
  c->P = P;
  c->Nc = Nc;
  c->hbody.assign(body.begin(), body.begin() + Nc);
  c->hcoff.assign(coff, coff + (P > 0 ? P + 1 : 0));
  CK(dalloc(c, &c->desc, sizeof(ParticleDesc) * desc.size()));
  CK(dalloc(c, &c->cbody, sizeof(float4) * body.size()));
  CK(copy_now(c, c->desc, desc.data(), sizeof(ParticleDesc) * desc.size()));
  CK(copy_now(c, c->cbody, body.data(), sizeof(float4) * body.size()));
  rwmi_status s = alloc_particles(c);
  if (s != RWMI_OK) return s;
  s = ensure_force_series(c);
  if (s != RWMI_OK) return s;
  drop_graphs(c);
  s = build_current_frame(c);
  if (s != RWMI_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_set_metaballs", e_);
}

RWMI_API void rwmi_dem_defaults(rwmi_dem_config* cfg) {
  if (!cfg) return;
  *cfg = rwmi_dem_config{};
  cfg->kn = 200.0;
  cfg->substeps = 10;
  cfg->hydro = 1;
}

RWMI_API rwmi_status rwmi_set_dem(rwmi_ctx* c, const rwmi_dem_config* cfg, const double* density,
                                  const double* Rs, const double* vel, const double* spin) try {
  if (!c || !cfg) return RWMI_E_INVALID;
  GUARD(c);
  if (c->P < 1 || !density || !Rs) return fail(c, RWMI_E_INVALID, "rwmi_set_dem: no particles or null array");
  if (c->dem) return fail(c, RWMI_E_STATE, "rwmi_set_dem: the particles are free already");
  if (c->cfg.storage != RWMI_STORE_FP32_SHIFT && c->cfg.storage != RWMI_STORE_FP64_SHIFT)
    return fail(c, RWMI_E_INVALID, "rwmi_set_dem: needs storage 1 or 3");
  if (!(cfg->kn >= 0.0) || !(cfg->eta_n >= 0.0) || !(cfg->kt >= 0.0) || !(cfg->eta_t >= 0.0) || !(cfg->mu_s >= 0.0) ||
      !std::isfinite(cfg->kn + cfg->eta_n + cfg->kt + cfg->eta_t + cfg->mu_s) || cfg->substeps < 1 ||
      cfg->substeps > 100000 || (cfg->hydro != 0 && cfg->hydro != 1))
    return fail(c, RWMI_E_INVALID, "rwmi_set_dem: bad contact law or substeps");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(cfg->gravity[a])) return fail(c, RWMI_E_INVALID, "rwmi_set_dem: non-finite gravity");
  const int P = c->P;
  std::vector<ParticleDesc> desc((size_t)P);
  CK(copy_now(c, desc.data(), c->desc, sizeof(ParticleDesc) * desc.size()));
  std::vector<double> st((size_t)13 * P, 0.0);
  for (int p = 0; p < P; ++p) {
    const ParticleDesc& d = desc[p];
    if (d.c1 - d.c0 > DEM_MAX_CP) return fail(c, RWMI_E_INVALID, "rwmi_set_dem: more than 16 control points");
    if (!(density[p] > 0.0) || !std::isfinite(density[p]) || !(Rs[p] > 0.0) || !std::isfinite(Rs[p]))
      return fail(c, RWMI_E_INVALID, "rwmi_set_dem: need density > 0 and R_s > 0");
    // the prescribed motion at the current time gives the start
    double s = 0.0, cdt = 0.0;
    if (d.period > 0.0) {
      const double th = 2.0 * 3.141592653589793 * (double)c->t / d.period + d.phase;
      s = std::sin(th);
      cdt = std::cos(th) * 2.0 * 3.141592653589793 / d.period;
    }
    double* q = st.data() + 13 * (size_t)p;
    for (int a = 0; a < 3; ++a) {
      q[a] = d.period > 0.0 ? d.org[a] + d.amp[a] * s : d.org[a];
      q[7 + a] = vel ? vel[3 * p + a] : d.amp[a] * cdt;
      q[10 + a] = spin ? spin[3 * p + a] : d.omega[a];
      if (!std::isfinite(q[7 + a]) || !std::isfinite(q[10 + a]))
        return fail(c, RWMI_E_INVALID, "rwmi_set_dem: non-finite velocity or spin");
    }
    q[3] = 1.0;
  }
  CK(dalloc(c, &c->dem_d, sizeof(double) * dem_doubles((size_t)P)));
  CK(dalloc(c, &c->dem_b, dem_bytes((size_t)P)));
  CK(cudaMemsetAsync(c->dem_d, 0, sizeof(double) * dem_doubles((size_t)P), c->stream));
  CK(cudaMemsetAsync(c->dem_b, 0, dem_bytes((size_t)P), c->stream));
  c->demcfg = *cfg;
  DemArgs a = dem_args(c, (int)(c->t & 1));
  {
    CallScratch<double> dens(c);
    CallScratch<unsigned long long> sums(c);
    CK(dalloc(c, &dens.p, sizeof(double) * (size_t)P));
    CK(dalloc(c, &sums.p, sizeof(unsigned long long) * 10 * (size_t)P));
    CK(cudaMemsetAsync(sums.p, 0, sizeof(unsigned long long) * 10 * (size_t)P, c->stream));
    CK(copy_now(c, a.st, st.data(), sizeof(double) * st.size()));
    CK(copy_now(c, dens.p, density, sizeof(double) * (size_t)P));
    CK(copy_now(c, const_cast<double*>(a.Rs), Rs, sizeof(double) * (size_t)P));
    launch_dem_mass(a, sums.p, dens.p, const_cast<double*>(a.mass), const_cast<double*>(a.Ib), dem_props(c),
                    c->cbody, c->stream);
  }
  const std::vector<float4> old_body = c->hbody;
  // the recentred body frames: host copy and bound radii
  CK(copy_now(c, c->hbody.data(), c->cbody, sizeof(float4) * c->hbody.size()));
  bool ok = true;
  std::vector<double> props((size_t)10 * P);
  CK(copy_now(c, props.data(), dem_props(c), sizeof(double) * props.size()));
  for (int p = 0; p < P; ++p) {
    ParticleDesc& d = desc[p];
    d.rb = bound_radius(c->hbody.data(), d.c0, d.c1);
    double reach = 0.0;   // validation only (the kernel forms the zoom)
    for (int i = d.c0; i < d.c1; ++i) {
      const float4 b = c->hbody[i];
      reach = std::max(reach, std::sqrt((double)b.x * b.x + (double)b.y * b.y + (double)b.z * b.z) +
                                  std::sqrt((double)b.w));
    }
    ok = ok && Rs[p] < reach && props[10 * p] > 0.0;
  }
  if (!ok) {   // restore the body frames: the context stays as it was
    c->hbody = old_body;
    CK(copy_now(c, c->cbody, old_body.data(), sizeof(float4) * old_body.size()));
    dfree(c, c->dem_d);
    dfree(c, c->dem_b);
    c->dem_d = nullptr;
    c->dem_b = nullptr;
    return fail(c, RWMI_E_INVALID, "rwmi_set_dem: need 0 < R_s < max |c_i - c_m| + sqrt(k_i) and a non-empty shape");
  }
  CK(copy_now(c, c->desc, desc.data(), sizeof(ParticleDesc) * desc.size()));
  a = dem_args(c, (int)(c->t & 1));
  launch_dem_init(a, c->stream);
  c->dem = true;
  drop_graphs(c);
  rwmi_status r = build_current_frame(c);
  if (r != RWMI_OK) return r;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_set_dem", e_);
}

RWMI_API rwmi_status rwmi_particle_mass(rwmi_ctx* c, double* out) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  if (!c->dem) return fail(c, RWMI_E_STATE, "rwmi_particle_mass: no free DEM (rwmi_set_dem)");
  CK(copy_now(c, out, dem_props(c), sizeof(double) * 10 * (size_t)c->P));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_particle_mass", e_);
}

RWMI_API rwmi_status rwmi_particle_state(rwmi_ctx* c, double* out) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  if (!c->dem) return fail(c, RWMI_E_STATE, "rwmi_particle_state: no free DEM (rwmi_set_dem)");
  CK(copy_now(c, out, c->dem_d, sizeof(double) * 13 * (size_t)c->P));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_particle_state", e_);
}

RWMI_API rwmi_status rwmi_set_particle_state(rwmi_ctx* c, const double* state) try {
  if (!c || !state) return RWMI_E_INVALID;
  GUARD(c);
  if (!c->dem) return fail(c, RWMI_E_STATE, "rwmi_set_particle_state: no free DEM (rwmi_set_dem)");
  for (size_t m = 0; m < (size_t)13 * c->P; ++m)
    if (!std::isfinite(state[m])) return fail(c, RWMI_E_INVALID, "rwmi_set_particle_state: non-finite value");
  CK(copy_now(c, c->dem_d, state, sizeof(double) * 13 * (size_t)c->P));
  launch_dem_init(dem_args(c, (int)(c->t & 1)), c->stream);   // zoom (unchanged) and reach cache
  rwmi_status r = build_current_frame(c);
  if (r != RWMI_OK) return r;
  CK(cudaStreamSynchronize(c->stream));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_set_particle_state", e_);
}

RWMI_API rwmi_status rwmi_seed_walkers(rwmi_ctx* c, int64_t n, const double lo[3], const double hi[3]) try {
  if (!c || !lo || !hi) return RWMI_E_INVALID;
  GUARD(c);
  if (n < 0 || n > 0x7fffffffLL) return fail(c, RWMI_E_INVALID, "rwmi_seed_walkers: 0 <= n < 2^31");
  for (int a = 0; a < 3; ++a)
    if (!(lo[a] >= 0.0) || !(hi[a] <= (double)c->n[a]) || !(lo[a] <= hi[a]))
      return fail(c, RWMI_E_INVALID, "rwmi_seed_walkers: box must lie in [0, n] per axis");
  rwmi_status s = alloc_walkers(c, n);
  if (s != RWMI_OK) return s;
  CK(cudaMemcpyAsync(c->status_seen, c->status, sizeof(unsigned long long) * ST_COUNT,
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const unsigned long long before = c->status_seen[ST_SEED_FAIL];
  launch_seed(c->g, particle_set(c), brick_set(c, (int)(c->t & 1)), c->pos[0], c->x0[0], n, lo, hi,
              (uint32_t)c->seed, (uint32_t)(c->seed >> 32), c->status, c->stream);
  c->launches++;
  CK(cudaGetLastError());
  unsigned long long st[ST_COUNT];
  CK(cudaMemcpyAsync(st, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->status_seen[ST_SEED_FAIL] = st[ST_SEED_FAIL];
  if (st[ST_SEED_FAIL] > before)
    return fail(c, RWMI_W_SEED, "rwmi_seed_walkers: some walkers found no free point in 1000 draws");
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_seed_walkers", e_);
}

RWMI_API rwmi_status rwmi_set_walkers(rwmi_ctx* c, int64_t n, const float* pos) try {
  if (!c || (n > 0 && !pos)) return RWMI_E_INVALID;
  GUARD(c);
  if (n < 0 || n > 0x7fffffffLL) return fail(c, RWMI_E_INVALID, "rwmi_set_walkers: 0 <= n < 2^31");
  std::vector<float> host;
  const float* src = pos;
  if (n > 0 && !is_device_ptr(pos)) {
    for (int64_t w = 0; w < n; ++w)
      for (int a = 0; a < 3; ++a) {
        const float v = pos[3 * w + a];
        if (!std::isfinite(v) || (c->g.wall[a] && (v < 0.0f || v > (float)c->n[a])))
          return fail(c, RWMI_E_INVALID, "rwmi_set_walkers: position outside the walls or not finite");
      }
  }
  rwmi_status s = alloc_walkers(c, n);
  if (s != RWMI_OK) return s;
  if (n == 0) return RWMI_OK;
  s = ensure_scratch(c, sizeof(float) * 3 * (size_t)n);
  if (s != RWMI_OK) return s;
  CK(cudaMemcpyAsync(c->scratch, src, sizeof(float) * 3 * (size_t)n, cudaMemcpyDefault, c->stream));
  launch_set_walkers((const float*)c->scratch, c->pos[0], c->x0[0], n, c->stream);
  c->launches++;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_set_walkers", e_);
}

RWMI_API rwmi_status rwmi_step(rwmi_ctx* c, int32_t n) try {
  if (!c || n < 0) return RWMI_E_INVALID;
  GUARD(c);
  c->stepped = true;
  const int64_t L = chunk_length(c);
  const bool graphs = c->cfg.use_graphs && L <= SEGMENT_MAX;
  // Runs of steps ("segments") of up to G steps, G the largest multiple of the chunk L within
  // SEGMENT_MAX: a long run repeats one captured segment, and any shorter run (or remainder) is
  // one captured segment too. Each segment ends by joining the walker stream, which exposes
  // one walker pass, so fewer and longer segments overlap more of the step.
  const int64_t G = graphs ? (SEGMENT_MAX / L) * L : 1;
  while (n > 0) {
    const int64_t k = std::min<int64_t>(n, graphs ? G - c->t % L : n);
    n -= (int32_t)k;
    const GraphKey key{c->fcur, c->pcur, c->t % L, k};
    auto it = graphs ? c->graphs.find(key) : c->graphs.end();
    if (graphs && it != c->graphs.end()) {
      CK(cudaGraphLaunch(it->second.exec, c->stream));
      c->launches += it->second.launches;
      advance_mirrors(c, k);
    } else if (graphs && c->graphs.size() < GRAPH_CACHE_MAX) {
      const int64_t l0 = c->launches;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      for (int64_t s = 0; s < k; ++s) enqueue_step(c, s == k - 1);   // sums on the run's last step
      segment_end(c);
      cudaGraph_t graph = nullptr;
      CK(cudaStreamEndCapture(c->stream, &graph));
      GraphEntry e;
      cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(ie);
      e.launches = c->launches - l0;
      c->graphs[key] = e;
      CK(cudaGraphLaunch(e.exec, c->stream));   // mirrors already advanced while capturing
    } else {   // eager; as in a captured run, the FP64 sums only on the run's last step
      for (int64_t s = 0; s < k; ++s) enqueue_step(c, s == k - 1);
      segment_end(c);
    }
  }
  CK(cudaGetLastError());
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_step", e_);
}

RWMI_API rwmi_status rwmi_step_timed(rwmi_ctx* c, int32_t n, double* phase_ms) try {
  if (!c || n < 0 || !phase_ms) return RWMI_E_INVALID;
  GUARD(c);
  c->stepped = true;
  for (int k = 0; k < 2 * RWMI_NPHASE; ++k)
    if (!c->ev[k]) CK(cudaEventCreate(&c->ev[k]));
  c->timing = true;
  for (int32_t s = 0; s < n; ++s) {
    enqueue_step(c, s == n - 1);   // as in a replayed chunk: the sums on the last step only
    segment_end(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      c->timing = false;
      CK(e);
    }
    for (int ph = 0; ph < RWMI_NPHASE; ++ph) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, c->ev[2 * ph], c->ev[2 * ph + 1]) == cudaSuccess) phase_ms[ph] += ms;
    }
  }
  c->timing = false;
  CK(cudaGetLastError());
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_step_timed", e_);
}

RWMI_API rwmi_status rwmi_autotune(rwmi_ctx* c, int32_t* chosen) try {
  if (!c) return RWMI_E_INVALID;
  GUARD(c);
  const int tp = (int)(c->t & 1);
  const size_t acc_n = (size_t)(6 * c->P + 4 * RED_SLOTS);
  rwmi_status s = ensure_scratch(c, sizeof(double) * acc_n);   // throw-away force/mass sums
  if (s != RWMI_OK) return s;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int cand[3] = {64, 128, 256};
  float best_ms = 1e30f;
  int best = 256;
  IbbArgs ia;
  const bool ibb = c->cfg.coupling == 1 && c->P > 0;
  if (ibb) {   // node classes of this time (no refilling: the step itself redoes them)
    launch_nodes(c->cfg.q, c->cfg.storage, c->g, particle_set(c), brick_set(c, tp), c->node[tp ^ 1], c->node[tp],
                 c->f[c->fcur], c->cfg.rho0, false, c->stream);
    c->launches++;
    ia.nodes = c->node[tp];
    ia.uprev = reinterpret_cast<const float4*>(c->u[tp ^ 1]);
    ia.desc = c->desc;
    launch_ibb_links(c->cfg.q, c->cfg.storage, c->g, brick_set(c, tp), c->node[tp], c->ibl, tp, c->desc,
                     c->f[c->fcur], c->u[tp ^ 1], c->cfg.rho0, c->status, c->nsm, c->stream);
    c->launches += 2;
    ia.base = c->ibl.base;
    ia.word = c->ibl.word;
    ia.q = c->ibl.q;
    ia.g = c->ibl.g;
    ia.cap = c->ibl.cap;
  }
  for (int k = 0; k < 3; ++k) {
    for (int rep = 0; rep < 6; ++rep) {
      if (rep == 1) cudaEventRecord(e0, c->stream);
      launch_lbm(c->cfg.q, c->cfg.storage, false, c->g, c->f[c->fcur], c->f[c->fcur ^ 1], c->u[c->t & 1], c->solid[c->t & 1],
                 brick_set(c, tp), c->tau, c->cfg.rho0, (double*)c->scratch + 6 * c->P,
                 (double*)c->scratch, c->status, c->stream, cand[k], ibb ? &ia : nullptr);
      c->launches++;
    }
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      CK(e);
    }
    if (ms < best_ms) { best_ms = ms; best = cand[k]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ibb) CK(cudaMemsetAsync(c->ibl.count, 0, sizeof(unsigned int) * 4, c->stream));   // the step appends anew
  CK(cudaGetLastError());
  c->cfg.lbm_block = best;
  drop_graphs(c);
  if (chosen) *chosen = best;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_autotune", e_);
}

RWMI_API rwmi_status rwmi_query(rwmi_ctx* c) try {
  if (!c) return RWMI_E_INVALID;
  GUARD(c);
  const cudaError_t e = cudaStreamQuery(c->stream);
  if (e == cudaErrorNotReady) return RWMI_BUSY;
  CK(e);
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_query", e_);
}

RWMI_API rwmi_status rwmi_footprint(const int32_t dims[3], int32_t q, int32_t storage, int64_t n_walkers,
                                    int32_t n_particles, int32_t n_centers, uint64_t* bytes) try {
  if (!dims || !bytes || (q != 15 && q != 19) || storage < 0 || storage > 3 || n_walkers < 0 ||
      n_particles < 0 || n_centers < 0)
    return RWMI_E_INVALID;
  uint64_t ncell = 1, nbrick = 1;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return RWMI_E_INVALID;
    ncell *= (uint64_t)dims[a];
    nbrick *= (uint64_t)((dims[a] + BRICK - 1) / BRICK);
  }
  const uint64_t pad = (ncell + 64) / 64 * 64, sb = storage_bytes(storage), P = (uint64_t)n_particles,
                 Nc = (uint64_t)n_centers, N = (uint64_t)n_walkers;
  uint64_t b = 2 * (uint64_t)q * pad * sb;                     // populations A/B
  b += 2 * 16 * pad + 2 * 2 * ncell + 2 * 2 * ncell + 8 * ncell + 4 * (ncell / 2048 + 2);   // (u, rho), solid, nodes, counts/offsets, scan
  b += 2 * (4 * (nbrick + BWORD_EXTRA) + 2 * MAXC * nbrick + 4 * nbrick) + 2 * 8 * nbrick;   // bricks, masks
  b += 100 * N;                                                // pos, x0 (A/B), rank, resolve list
  b += 2 * (48 + 80) * P + 2 * 16 * Nc + sizeof(ParticleDesc) * P + 16 * Nc + 2 * 8 * (6 * P + 4 * RED_SLOTS);
  b += (uint64_t)SERIES_ROWS * SERIES_COLS * 8 + 4096;         // moment series, counters
  *bytes = b;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return RWMI_E_OOM;
}

RWMI_API rwmi_status rwmi_sync(rwmi_ctx* c) try {
  if (!c) return RWMI_E_INVALID;
  GUARD(c);
  CK(cudaStreamSynchronize(c->stream));
  unsigned long long st[ST_COUNT];
  CK(copy_now(c, st, c->status, sizeof(st)));
  rwmi_status r = RWMI_OK;
  if (st[ST_IBB_OVERFLOW] > c->status_seen[ST_IBB_OVERFLOW])
    r = fail(c, RWMI_E_OOM, "IBB link list and overflow slots full: a step ran with links missing");
  else if (st[ST_TMA_TIMEOUT] > c->status_seen[ST_TMA_TIMEOUT])
    r = fail(c, RWMI_E_TIMEOUT, "a bounded wait for a TMA copy gave up (the LBM update is incomplete)");
  else if (st[ST_NONFINITE] > c->status_seen[ST_NONFINITE]) r = fail(c, RWMI_E_NONFINITE, "non-finite walker velocity");
  else if (st[ST_BISECT_FAIL] > c->status_seen[ST_BISECT_FAIL] || st[ST_REFILL_FAIL] > c->status_seen[ST_REFILL_FAIL])
    r = fail(c, RWMI_W_BISECT, "Algorithm 1 or the refill found no surface point for some walker");
  std::memcpy(c->status_seen, st, sizeof(st));
  return r;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_sync", e_);
}

RWMI_API rwmi_status rwmi_time(rwmi_ctx* c, int64_t* t) try {
  if (!c || !t) return RWMI_E_INVALID;
  GUARD(c);
  *t = c->t;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_time", e_);
}

RWMI_API rwmi_status rwmi_info(rwmi_ctx* c, int64_t out[8]) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  const int64_t v[8] = {c->n[0], c->n[1], c->n[2], c->cfg.q, c->cfg.storage, c->nw, c->P, c->t};
  std::memcpy(out, v, sizeof(v));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_info", e_);
}

RWMI_API rwmi_status rwmi_concentration(rwmi_ctx* c, uint32_t* out) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  if (c->binned_t != c->t) {
    CK(cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * (size_t)c->ncell, c->stream));
    launch_histogram(c->g, c->pos[c->pcur], c->nw, c->counts, nullptr, c->stream);
    c->launches++;
    CK(cudaGetLastError());
    c->binned_t = c->t;
  }
  return copy_out(c, out, c->counts, sizeof(uint32_t) * (size_t)c->ncell);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_concentration", e_);
}

RWMI_API rwmi_status rwmi_walker_moments(rwmi_ctx* c, double out[13]) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  launch_moments(c->pos[c->pcur], c->x0[c->pcur], c->nw, c->macc, c->mrow, 0, 1, c->d_T, 0, c->stream);
  c->launches += c->nw > 0 ? 2 : 1;
  CK(cudaGetLastError());
  return copy_out(c, out, c->mrow + 1, sizeof(double) * 13);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_walker_moments", e_);
}

RWMI_API rwmi_status rwmi_moment_series(rwmi_ctx* c, double* out, int32_t max_rows, int32_t* n_rows) try {
  if (!c || !out || !n_rows || max_rows < 0) return RWMI_E_INVALID;
  GUARD(c);
  const int64_t avail = std::min<int64_t>(c->series_rows, SERIES_ROWS);
  const int64_t take = std::min<int64_t>(avail, max_rows);
  std::vector<double> ring((size_t)SERIES_ROWS * SERIES_COLS);
  CK(cudaStreamSynchronize(c->stream));
  CK(copy_now(c, ring.data(), c->series, sizeof(double) * ring.size()));
  std::vector<double> rows((size_t)take * SERIES_COLS);
  const int64_t first = c->series_rows - take;
  for (int64_t r = 0; r < take; ++r)
    std::memcpy(&rows[(size_t)r * SERIES_COLS], &ring[(size_t)((first + r) % SERIES_ROWS) * SERIES_COLS],
                sizeof(double) * SERIES_COLS);
  if (take > 0) CK(copy_now(c, out, rows.data(), sizeof(double) * rows.size()));
  *n_rows = (int32_t)take;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_moment_series", e_);
}

RWMI_API rwmi_status rwmi_velocity(rwmi_ctx* c, float* out) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  rwmi_status s = ensure_scratch(c, sizeof(float) * 3 * (size_t)c->ncell);
  if (s != RWMI_OK) return s;
  launch_velocity_aos(c->g, c->u[(c->t + 1) & 1], (float*)c->scratch, c->stream);
  c->launches++;
  CK(cudaGetLastError());
  return copy_out(c, out, c->scratch, sizeof(float) * 3 * (size_t)c->ncell);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_velocity", e_);
}

RWMI_API rwmi_status rwmi_density(rwmi_ctx* c, float* out) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  rwmi_status s = ensure_scratch(c, sizeof(float) * (size_t)c->ncell);
  if (s != RWMI_OK) return s;
  launch_density(c->cfg.q, c->cfg.storage, c->g, c->f[c->fcur], c->cfg.rho0, (float*)c->scratch, c->stream);
  c->launches++;
  CK(cudaGetLastError());
  return copy_out(c, out, c->scratch, sizeof(float) * (size_t)c->ncell);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_density", e_);
}

RWMI_API rwmi_status rwmi_populations(rwmi_ctx* c, double* out) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  const size_t bytes = sizeof(double) * (size_t)c->cfg.q * (size_t)c->ncell;
  rwmi_status s = ensure_scratch(c, bytes);
  if (s != RWMI_OK) return s;
  launch_populations_f64(c->cfg.q, c->cfg.storage, c->g, c->f[c->fcur], c->cfg.rho0,
                         (double*)c->scratch, c->stream);
  c->launches++;
  CK(cudaGetLastError());
  return copy_out(c, out, c->scratch, bytes);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_populations", e_);
}

RWMI_API rwmi_status rwmi_lattice(rwmi_ctx* c, int32_t* e, double* w, int32_t* q) try {
  if (!c) return RWMI_E_INVALID;
  GUARD(c);
  if (q) *q = c->cfg.q;
  if (e && w) lattice_table(c->cfg.q, e, w);
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_lattice", e_);
}

RWMI_API rwmi_status rwmi_solid(rwmi_ctx* c, int32_t* count, int32_t* owner) try {
  if (!c || !count || !owner) return RWMI_E_INVALID;
  GUARD(c);
  const int par = (int)(c->t & 1);
  const size_t bytes = sizeof(int32_t) * 2 * (size_t)c->ncell;
  rwmi_status s = ensure_scratch(c, bytes);
  if (s != RWMI_OK) return s;
  int32_t* tmp = (int32_t*)c->scratch;   // the current time was rasterised by the last step / set-up
  if (c->cfg.coupling == 1 && c->P > 0) {
    // IBB steps rasterise bricks and walker masks only: the counts of the current time are formed
    // here, from its bricks (intact until the next step), by a full raster with a reset work
    // counter (it rewrites the same walker masks)
    CK(cudaMemsetAsync(c->bword[par] + c->nbrick + 1, 0, sizeof(uint32_t), c->stream));
    launch_raster(c->g, particle_set(c), brick_set(c, par), c->solid[par], c->status, c->nsm, c->stream, true);
    c->launches++;
  }
  launch_unpack_solid(c->g, c->solid[par], c->bword[par], tmp, tmp + c->ncell, c->stream);
  c->launches++;
  CK(cudaGetLastError());
  s = copy_out(c, count, tmp, sizeof(int32_t) * (size_t)c->ncell);
  if (s != RWMI_OK) return s;
  return copy_out(c, owner, tmp + c->ncell, sizeof(int32_t) * (size_t)c->ncell);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_solid", e_);
}

RWMI_API rwmi_status rwmi_nodes(rwmi_ctx* c, int32_t* node) try {
  if (!c || !node) return RWMI_E_INVALID;
  GUARD(c);
  const int par = (int)(c->t & 1);
  const size_t n = (size_t)c->ncell;
  rwmi_status s = ensure_scratch(c, (sizeof(uint16_t) + sizeof(int32_t)) * n + 256);
  if (s != RWMI_OK) return s;
  uint16_t* tmp = (uint16_t*)c->scratch;
  if (c->P > 0) {
    launch_nodes(c->cfg.q, c->cfg.storage, c->g, particle_set(c), brick_set(c, par), tmp, tmp, c->f[c->fcur],
                 c->cfg.rho0, false, c->stream);
    c->launches++;
  } else {
    CK(cudaMemsetAsync(tmp, 0, sizeof(uint16_t) * n, c->stream));
  }
  std::vector<uint16_t> h(n);
  CK(copy_now(c, h.data(), tmp, sizeof(uint16_t) * n));
  std::vector<int32_t> o(n);
  for (size_t k = 0; k < n; ++k) o[k] = h[k];
  CK(copy_now(c, node, o.data(), sizeof(int32_t) * n));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_nodes", e_);
}

RWMI_API rwmi_status rwmi_mass_momentum(rwmi_ctx* c, double out[4]) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (c->t > 0) {
    std::vector<double> slots((size_t)4 * RED_SLOTS);
    rwmi_status s = copy_out(c, slots.data(), c->acc[(c->t - 1) & 1] + 6 * c->P, sizeof(double) * slots.size());
    if (s != RWMI_OK) return s;
    for (int k = 0; k < RED_SLOTS; ++k)
      for (int m = 0; m < 4; ++m) v[m] += slots[4 * k + m];
  }
  out[0] = (double)c->ncell * c->cfg.rho0 + v[0];
  out[1] = v[1]; out[2] = v[2]; out[3] = v[3];
  if (!std::isfinite(out[0])) return fail(c, RWMI_E_NONFINITE, "non-finite mass sum");
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_mass_momentum", e_);
}

RWMI_API rwmi_status rwmi_particle_forces(rwmi_ctx* c, double* out) try {
  if (!c || (!out && c->P > 0)) return RWMI_E_INVALID;
  GUARD(c);
  if (c->P == 0) return RWMI_OK;
  if (c->t == 0) {
    std::vector<double> z((size_t)6 * c->P, 0.0);
    CK(copy_now(c, out, z.data(), sizeof(double) * z.size()));
    return RWMI_OK;
  }
  return copy_out(c, out, c->acc[(c->t - 1) & 1], sizeof(double) * 6 * (size_t)c->P);
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_particle_forces", e_);
}

RWMI_API rwmi_status rwmi_force_series(rwmi_ctx* c, double* out, int32_t max_rows, int32_t* n_rows) try {
  if (!c || !out || !n_rows || max_rows < 0) return RWMI_E_INVALID;
  GUARD(c);
  if (c->P == 0 || c->cfg.force_interval == 0 || !c->fseries)
    return fail(c, RWMI_E_INVALID, "rwmi_force_series: no particles or force_interval 0");
  const size_t cols = 1 + 6 * (size_t)c->P;
  const int64_t avail = std::min<int64_t>(c->fseries_rows, FORCE_ROWS);
  const int64_t take = std::min<int64_t>(avail, max_rows);
  CK(cudaStreamSynchronize(c->stream));
  // the newest `take` rows of the ring, oldest first: at most two contiguous pieces
  const int64_t first = (c->fseries_rows - take) % FORCE_ROWS;
  const int64_t n1 = std::min<int64_t>(take, FORCE_ROWS - first);
  if (n1 > 0) CK(copy_now(c, out, c->fseries + (size_t)first * cols, sizeof(double) * (size_t)n1 * cols));
  if (take > n1) CK(copy_now(c, out + (size_t)n1 * cols, c->fseries, sizeof(double) * (size_t)(take - n1) * cols));
  *n_rows = (int32_t)take;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_force_series", e_);
}

RWMI_API rwmi_status rwmi_walkers(rwmi_ctx* c, float* out, float* x0) try {
  if (!c || (!out && c->nw > 0)) return RWMI_E_INVALID;
  GUARD(c);
  if (c->nw == 0) return RWMI_OK;
  rwmi_status s = copy_out(c, out, c->pos[c->pcur], sizeof(float4) * (size_t)c->nw);
  if (s != RWMI_OK) return s;
  if (x0) {
    const cudaMemcpyKind k = is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpy2DAsync(x0, 3 * sizeof(float), c->x0[c->pcur], sizeof(float4), 3 * sizeof(float),
                         (size_t)c->nw, k, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_walkers", e_);
}

RWMI_API rwmi_status rwmi_counters(rwmi_ctx* c, int64_t out[12]) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  CK(cudaStreamSynchronize(c->stream));
  unsigned long long st[ST_COUNT];
  CK(copy_now(c, st, c->status, sizeof(st)));
  for (int m = 0; m < 8; ++m) out[m] = (int64_t)st[m];
  out[8] = (int64_t)st[ST_NONFINITE];
  out[9] = (int64_t)st[ST_FAST_SPEED];
  out[10] = (int64_t)st[ST_RESOLVED];
  out[11] = (int64_t)st[ST_RASTER_QUEUED];
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_counters", e_);
}

RWMI_API rwmi_status rwmi_save(rwmi_ctx* c, const char* path) try {
  if (!c || !path) return RWMI_E_INVALID;
  GUARD(c);
  CK(cudaStreamSynchronize(c->stream));
  const size_t pop = (size_t)c->cfg.q * c->g.ncell_pad * storage_bytes(c->cfg.storage);
  std::vector<char> f(pop);
  std::vector<float4> p((size_t)c->nw), q((size_t)c->nw);
  CK(copy_now(c, f.data(), c->f[c->fcur], pop));
  if (c->nw) {
    CK(copy_now(c, p.data(), c->pos[c->pcur], sizeof(float4) * p.size()));
    CK(copy_now(c, q.data(), c->x0[c->pcur], sizeof(float4) * q.size()));
  }
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(c, RWMI_E_INVALID, std::string("rwmi_save: cannot open ") + path);
  const int64_t hdr[10] = {(int64_t)CKPT_MAGIC, c->cfg.q, c->cfg.storage, c->n[0], c->n[1], c->n[2],
                           c->nw, c->t, c->P, c->Nc};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, fp) == 1 && std::fwrite(f.data(), 1, pop, fp) == pop;
  if (c->nw) ok = ok && std::fwrite(p.data(), sizeof(float4), p.size(), fp) == p.size() &&
                  std::fwrite(q.data(), sizeof(float4), q.size(), fp) == q.size();
  if (c->dem && ok) {   // free DEM: state, parameters, contact memory and flags
    std::vector<double> dd(dem_doubles((size_t)c->P));
    std::vector<unsigned char> db(dem_bytes((size_t)c->P));
    if (copy_now(c, dd.data(), c->dem_d, sizeof(double) * dd.size()) != cudaSuccess ||
        copy_now(c, db.data(), c->dem_b, db.size()) != cudaSuccess) {
      std::fclose(fp);
      return fail(c, RWMI_E_CUDA, "rwmi_save: reading the DEM state failed");
    }
    const int64_t dh[2] = {(int64_t)CKPT_DEM_MAGIC, c->P};
    ok = std::fwrite(dh, sizeof(dh), 1, fp) == 1 && std::fwrite(&c->demcfg, sizeof(c->demcfg), 1, fp) == 1 &&
         std::fwrite(dd.data(), sizeof(double), dd.size(), fp) == dd.size() &&
         std::fwrite(db.data(), 1, db.size(), fp) == db.size();
  }
  ok = (std::fclose(fp) == 0) && ok;
  if (!ok) return fail(c, RWMI_E_INVALID, "rwmi_save: write failed");
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_save", e_);
}

RWMI_API rwmi_status rwmi_load(rwmi_ctx* c, const char* path) try {
  if (!c || !path) return RWMI_E_INVALID;
  GUARD(c);
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(c, RWMI_E_INVALID, std::string("rwmi_load: cannot open ") + path);
  int64_t hdr[10];
  if (std::fread(hdr, sizeof(hdr), 1, fp) != 1 || hdr[0] != (int64_t)CKPT_MAGIC || hdr[1] != c->cfg.q ||
      hdr[2] != c->cfg.storage || hdr[3] != c->n[0] || hdr[4] != c->n[1] || hdr[5] != c->n[2] ||
      hdr[8] != c->P || hdr[9] != c->Nc || hdr[6] < 0 || hdr[7] < 0) {
    std::fclose(fp);
    return fail(c, RWMI_E_INVALID, "rwmi_load: checkpoint does not match this context");
  }
  const size_t pop = (size_t)c->cfg.q * c->g.ncell_pad * storage_bytes(c->cfg.storage);
  const int64_t nw = hdr[6];
  // A corrupt walker count is refused before anything is allocated: the file must hold it.
  const long here = std::ftell(fp);
  const long size = std::fseek(fp, 0, SEEK_END) == 0 ? std::ftell(fp) : -1L;
  if (here < 0 || size < here || std::fseek(fp, here, SEEK_SET) != 0 || nw > 0x7fffffffLL ||
      (uint64_t)(size - here) < (uint64_t)pop + 2 * sizeof(float4) * (uint64_t)nw) {
    std::fclose(fp);
    return fail(c, RWMI_E_INVALID, "rwmi_load: truncated checkpoint or corrupt walker count");
  }
  std::vector<char> f(pop);
  std::vector<float4> p((size_t)nw), q((size_t)nw);
  bool ok = std::fread(f.data(), 1, pop, fp) == pop;
  if (nw) ok = ok && std::fread(p.data(), sizeof(float4), p.size(), fp) == p.size() &&
               std::fread(q.data(), sizeof(float4), q.size(), fp) == q.size();
  std::vector<double> dd;
  std::vector<unsigned char> db;
  rwmi_dem_config dcfg{};
  int64_t dh[2] = {0, 0};
  const bool has_dem = ok && std::fread(dh, sizeof(dh), 1, fp) == 1 && dh[0] == (int64_t)CKPT_DEM_MAGIC;
  if (has_dem) {
    dd.resize(dem_doubles((size_t)c->P));
    db.resize(dem_bytes((size_t)c->P));
    ok = dh[1] == c->P && std::fread(&dcfg, sizeof(dcfg), 1, fp) == 1 &&
         std::fread(dd.data(), sizeof(double), dd.size(), fp) == dd.size() &&
         std::fread(db.data(), 1, db.size(), fp) == db.size();
  }
  std::fclose(fp);
  if (!ok) return fail(c, RWMI_E_INVALID, "rwmi_load: truncated checkpoint");
  if (has_dem != c->dem)
    return fail(c, RWMI_E_INVALID, "rwmi_load: free-DEM checkpoints load into free-DEM contexts only");
  CK(cudaStreamSynchronize(c->stream));
  if (nw != c->nw) {
    rwmi_status s = alloc_walkers(c, nw);
    if (s != RWMI_OK) return s;
  }
  c->t = hdr[7];
  c->fcur = (int)(c->t & 1);
  c->pcur = 0;
  c->binned_t = -1;
  c->stepped = true;
  drop_graphs(c);
  CK(copy_now(c, c->f[c->fcur], f.data(), pop));
  if (nw) {
    CK(copy_now(c, c->pos[0], p.data(), sizeof(float4) * p.size()));
    CK(copy_now(c, c->x0[0], q.data(), sizeof(float4) * q.size()));
  }
  if (has_dem) {
    c->demcfg = dcfg;
    CK(copy_now(c, c->dem_d, dd.data(), sizeof(double) * dd.size()));
    CK(copy_now(c, c->dem_b, db.data(), db.size()));
  }
  CK(copy_now(c, c->d_T, &c->t, sizeof(int64_t)));
  c->t_base = c->t;
  CK(cudaMemsetAsync(c->wlist_n, 0, sizeof(unsigned int) * 2 * WLIST_STRIPES, c->stream));
  if (c->ibl.count) CK(cudaMemsetAsync(c->ibl.count, 0, sizeof(unsigned int) * 4, c->stream));
  rwmi_status s = build_current_frame(c);
  if (s != RWMI_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_load", e_);
}

RWMI_API rwmi_status rwmi_brick_stats(rwmi_ctx* c, int64_t out[4]) try {
  if (!c || !out) return RWMI_E_INVALID;
  GUARD(c);
  std::vector<uint32_t> w((size_t)c->nbrick + 1);
  CK(cudaStreamSynchronize(c->stream));
  CK(copy_now(c, w.data(), c->bword[c->t & 1], sizeof(uint32_t) * w.size()));
  int64_t rast = 0, walk = 0, mx = 0, over = 0;
  for (uint32_t b = 0; b < c->nbrick; ++b) {
    const int64_t nc = w[b] & 0xffffu;
    rast += (w[b] >> 16) ? 1 : 0;
    walk += nc ? 1 : 0;
    mx = std::max(mx, nc);
    over += nc > MAXC ? 1 : 0;
  }
  out[0] = rast; out[1] = walk; out[2] = mx; out[3] = over;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return api_exception(c, "rwmi_brick_stats", e_);
}

static rwmi_status batch_fail(rwmi_batch* b, rwmi_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return batch_fail(b, RWMI_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

RWMI_API void rwmi_batch_destroy(rwmi_batch* b);

namespace {

// A context runs in a fused batch when its step is the plain one of the hot path: partially
// saturated cells, prescribed particles, and the batch's velocity set, storage and intervals.
bool fusable(const rwmi_ctx* c, const rwmi_ctx* c0) {
  return c->cfg.coupling == 0 && !c->dem && c->cfg.force_interval == 0 && c->cfg.q == c0->cfg.q &&
         c->cfg.storage == c0->cfg.storage && c->cfg.sort_interval == c0->cfg.sort_interval &&
         c->cfg.moment_interval == c0->cfg.moment_interval;
}

void fused_drop_graphs(rwmi_batch* b) {
  for (auto& kv : b->fgraphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.args) cudaFreeAsync(kv.second.args, b->origin);
  }
  b->fgraphs.clear();
}

int64_t ceil_div(int64_t a, int64_t d) { return (a + d - 1) / d; }

// RWMI_BATCH_AUTO: fused launches where launch gaps dominate, i.e. for small domains. With a mean
// below 2^19 cells per context (a domain's LBM then runs for ~10 us, about two launch gaps) the
// fused form measured 2.7x faster than the branches for 256 domains of 16^3-48^3; for 64
// domains of 48^3-160^3 (mean 1.6 M cells) the branches were 10% faster, since each domain's
// phases then pipeline independently instead of waiting for every domain's.
bool fused_pays(const rwmi_batch* b) {
  int64_t cells = 0;
  for (const rwmi_ctx* c : b->ctxs) cells += c->ncell;
  return cells < (int64_t)b->ctxs.size() * (int64_t)(1 << 19);
}

// Block maps of every phase from the contexts' sizes and the batch's work split: each context
// gets the grid its own launch would take, except where the tiles set it (LBM block size, walker
// chunks per block, walkers per resolve block, bricks per raster block).
rwmi_status fused_build_maps(rwmi_batch* b) {
  std::vector<BlockMap> all;
  const rwmi_batch_tiles& tl = b->tiles;
  auto add = [&](int phase, auto blocks_of) {
    b->map_off[phase] = all.size();
    for (size_t d = 0; d < b->ctxs.size(); ++d) {
      const int nb = (int)blocks_of(b->ctxs[d]);
      for (int k = 0; k < nb; ++k) all.push_back(BlockMap{(int32_t)d, k, nb, 0});
    }
    b->map_n[phase] = all.size() - b->map_off[phase];
  };
  const bool sorts = b->ctxs[0]->cfg.sort_interval > 0, moments = b->ctxs[0]->cfg.moment_interval > 0;
  add(FP_CLEARB, [&](rwmi_ctx* c) { return clear_grid(c->nbrick + BWORD_EXTRA); });
  add(FP_POSE, [&](rwmi_ctx* c) { return c->P > 0 ? c->P : 1; });
  add(FP_RASTER, [&](rwmi_ctx* c) {
    return c->P > 0 ? std::min<int64_t>(std::max<int64_t>(ceil_div(c->nbrick, tl.raster_bricks_per_block), 1),
                                        raster_grid(c->nsm))
                    : 0;
  });
  add(FP_LBM, [&](rwmi_ctx* c) { return ceil_div(c->ncell, tl.lbm_block); });
  add(FP_WALK, [&](rwmi_ctx* c) { return c->nw > 0 ? ceil_div(ceil_div(c->nw, 256), tl.walker_chunks_per_block) : 0; });
  add(FP_RESOLVE, [&](rwmi_ctx* c) {
    return c->nw > 0 ? std::min<int64_t>(ceil_div(c->nw, tl.resolve_walkers_per_block), resolve_grid(c->nsm)) : 0;
  });
  add(FP_CLEARC, [&](rwmi_ctx* c) { return sorts && c->nw > 0 ? clear_grid((uint32_t)c->ncell) : 0; });
  add(FP_HIST, [&](rwmi_ctx* c) { return sorts && c->nw > 0 ? ceil_div(c->nw, 256) : 0; });
  add(FP_SCANR, [&](rwmi_ctx* c) { return sorts && c->nw > 0 ? (int64_t)scan_tiles((uint32_t)c->ncell) : 0; });
  add(FP_SCANT, [&](rwmi_ctx* c) { return sorts && c->nw > 0 ? 1 : 0; });
  add(FP_SCAND, [&](rwmi_ctx* c) { return sorts && c->nw > 0 ? (int64_t)scan_tiles((uint32_t)c->ncell) : 0; });
  add(FP_SCATTER, [&](rwmi_ctx* c) { return sorts && c->nw > 0 ? ceil_div(c->nw, 256) : 0; });
  add(FP_MOM, [&](rwmi_ctx* c) { return moments && c->nw > 0 ? moments_grid(c->nw) : 0; });
  add(FP_MOMFIN, [&](rwmi_ctx* c) { return moments ? 1 : 0; });
  add(FP_ADV, [&](rwmi_ctx*) { return 1; });
  if (b->maps) cudaFreeAsync(b->maps, b->origin);
  b->maps = nullptr;
  cudaError_t e = cudaMallocAsync(&b->maps, sizeof(BlockMap) * all.size(), b->origin);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->maps, all.data(), sizeof(BlockMap) * all.size(), cudaMemcpyHostToDevice, b->origin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
  if (e != cudaSuccess)
    return batch_fail(b, e == cudaErrorMemoryAllocation ? RWMI_E_OOM : RWMI_E_CUDA,
                      std::string("fused batch maps: ") + cudaGetErrorString(e));
  return RWMI_OK;
}

// Captures one chunk of L steps of every context as fused launches. The argument records of
// every step are formed on the host while the host mirrors advance, exactly as enqueue_step
// advances them, in its pipelined schedule: the raster of t+1 beside the LBM of t, and the
// walkers of t (with the sort and moments) on a third stream beside the fluid of t+1; the fluid
// of t+2 waits for the walkers of t, the last readers of the buffers of that time parity.
rwmi_status fused_capture(rwmi_batch* b, FusedGraph& fg) {
  const size_t ND = b->ctxs.size();
  const int64_t L = b->L;
  rwmi_ctx* c0 = b->ctxs[0];
  const int q = c0->cfg.q, storage = c0->cfg.storage;
  const size_t sz[FP_COUNT] = {clear_args_size(), pose_args_size(), raster_args_size(), lbm_args_size(q, storage),
                               walker_args_size(), walker_args_size(), clear_args_size(), hist_args_size(),
                               scan_args_size(), scan_args_size(), scan_args_size(), scatter_args_size(),
                               moments_args_size(), moments_args_size(), advance_args_size()};
  auto round16 = [](size_t v) { return (v + 15) / 16 * 16; };
  std::vector<std::vector<size_t>> off(L, std::vector<size_t>(FP_COUNT));
  size_t total = 0;
  for (int64_t s = 0; s < L; ++s)
    for (int p = 0; p < FP_COUNT; ++p) {
      off[s][p] = total;
      total += round16(sz[p] * ND);
    }
  std::vector<unsigned char> blob(total, 0);
  bool walls = false;
  for (rwmi_ctx* c : b->ctxs) walls = walls || c->g.wall[0] || c->g.wall[1] || c->g.wall[2];
  bool sort_at[64] = {}, mom_at[64] = {};
  for (int64_t s = 0; s < L; ++s) {
    for (size_t d = 0; d < ND; ++d) {
      rwmi_ctx* c = b->ctxs[d];
      const int tp = (int)(c->t & 1), tn = tp ^ 1;
      const int toff = (int)(c->t - c->t_base);
      const ParticleSet ps = particle_set(c);
      const uint32_t k0 = (uint32_t)c->seed, k1 = (uint32_t)(c->seed >> 32);
      auto rec = [&](int p) { return blob.data() + off[s][p] + sz[p] * d; };
      clear_args(rec(FP_CLEARB), c->bword[tn], c->nbrick + BWORD_EXTRA);
      pose_args(rec(FP_POSE), c->g, ps, brick_set(c, tn), c->d_T, toff + 1, c->cfg.body_force, c->cfg.force_period, 1,
                c->acc[tn], c->cfg.q, c->tau);
      raster_args(rec(FP_RASTER), c->g, ps, brick_set(c, tn), c->solid[tn], c->status);
      lbm_args(rec(FP_LBM), q, storage, c->g, c->f[c->fcur], c->f[c->fcur ^ 1], c->u[tp], c->solid[tp],
               brick_set(c, tp), c->tau, c->cfg.rho0, c->acc[tp] + 6 * c->P, c->acc[tp]);
      walker_args(rec(FP_WALK), c->g, ps, brick_set(c, tn), c->pos[c->pcur], c->nw, c->u[tp], c->d_T, toff, tp,
                  (float)c->D, k0, k1, c->status, c->wlist, c->wlist_n);
      std::memcpy(rec(FP_RESOLVE), rec(FP_WALK), sz[FP_WALK]);
      c->fcur ^= 1;
      c->t += 1;
      const bool sort = c->nw > 0 && c->cfg.sort_interval > 0 && c->t % c->cfg.sort_interval == 0;
      if (sort) {
        clear_args(rec(FP_CLEARC), c->counts, (uint32_t)c->ncell);
        hist_args(rec(FP_HIST), c->g, c->pos[c->pcur], c->nw, c->counts, c->rank);
        scan_args(rec(FP_SCANR), c->counts, c->offsets, c->bsums, (uint32_t)c->ncell);
        std::memcpy(rec(FP_SCANT), rec(FP_SCANR), sz[FP_SCANR]);
        std::memcpy(rec(FP_SCAND), rec(FP_SCANR), sz[FP_SCANR]);
        scatter_args(rec(FP_SCATTER), c->g, c->pos[c->pcur], c->x0[c->pcur], c->nw, c->offsets, c->rank,
                     c->pos[c->pcur ^ 1], c->x0[c->pcur ^ 1]);
        c->pcur ^= 1;
        c->binned_t = c->t;
      }
      const bool mom = c->cfg.moment_interval > 0 && c->t % c->cfg.moment_interval == 0;
      if (mom) {
        moments_args(rec(FP_MOM), c->pos[c->pcur], c->x0[c->pcur], c->nw, c->macc, c->series,
                     c->cfg.moment_interval, SERIES_ROWS, c->d_T, toff + 1);
        std::memcpy(rec(FP_MOMFIN), rec(FP_MOM), sz[FP_MOM]);
        c->series_rows++;
      }
      if (d == 0) { sort_at[s] = c->cfg.sort_interval > 0 && c->t % c->cfg.sort_interval == 0; mom_at[s] = mom; }
      if (s == L - 1) advance_args(rec(FP_ADV), c->d_T, L);
    }
  }
  for (rwmi_ctx* c : b->ctxs) c->t_base = c->t;
  cudaError_t e = cudaMallocAsync(&fg.args, total, b->origin);
  if (e == cudaSuccess) e = cudaMemcpyAsync(fg.args, blob.data(), total, cudaMemcpyHostToDevice, b->origin);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
  if (e != cudaSuccess)
    return batch_fail(b, e == cudaErrorMemoryAllocation ? RWMI_E_OOM : RWMI_E_CUDA,
                      std::string("fused batch arguments: ") + cudaGetErrorString(e));
  const unsigned char* dev = static_cast<const unsigned char*>(fg.args);
  auto A = [&](int64_t s, int p) { return (const void*)(dev + off[s][p]); };
  auto M = [&](int p) { return b->maps + b->map_off[p]; };
  auto N = [&](int p) { return (int)b->map_n[p]; };
  int64_t launches = 0;
  auto count = [&](int p) { launches += N(p) > 0 ? 1 : 0; };
  BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
  bool walk_rec[2] = {false, false};
  for (int64_t s = 0; s < L; ++s) {
    const int par = (int)(s & 1);   // every context is at an even time at the chunk start
    if (walk_rec[par]) cudaStreamWaitEvent(b->origin, b->walk_ev[par], 0);
    launch_clear_batched(A(s, FP_CLEARB), M(FP_CLEARB), N(FP_CLEARB), b->origin); count(FP_CLEARB);
    launch_pose_batched(A(s, FP_POSE), M(FP_POSE), N(FP_POSE), b->origin); count(FP_POSE);
    cudaEventRecord(b->fork2, b->origin);
    cudaStreamWaitEvent(b->side, b->fork2, 0);
    launch_raster_batched(A(s, FP_RASTER), M(FP_RASTER), N(FP_RASTER), b->side); count(FP_RASTER);
    cudaEventRecord(b->join2, b->side);
    // the FP64 sums on the chunk's last step, as in rwmi_step: the fused update-and-reduce pass
    // where the storage has one (same stored bits), else the update and a reduce-only pass
    const bool fuse = s == L - 1 && fused_storage(storage);
    launch_lbm_batched(q, storage, walls, fuse ? 2 : 0, A(s, FP_LBM), M(FP_LBM), N(FP_LBM), b->tiles.lbm_block,
                       b->origin);
    count(FP_LBM);
    if (s == L - 1 && !fuse) {
      launch_lbm_batched(q, storage, walls, 1, A(s, FP_LBM), M(FP_LBM), N(FP_LBM), b->tiles.lbm_block, b->origin);
      count(FP_LBM);
    }
    cudaStreamWaitEvent(b->origin, b->join2, 0);
    cudaEventRecord(b->fluid_ev, b->origin);
    cudaStreamWaitEvent(b->wst, b->fluid_ev, 0);
    cudaStream_t ws = b->wst;
    launch_walker_batched(A(s, FP_WALK), M(FP_WALK), N(FP_WALK), ws); count(FP_WALK);
    launch_resolve_batched(A(s, FP_RESOLVE), M(FP_RESOLVE), N(FP_RESOLVE), ws); count(FP_RESOLVE);
    if (sort_at[s]) {
      launch_clear_batched(A(s, FP_CLEARC), M(FP_CLEARC), N(FP_CLEARC), ws); count(FP_CLEARC);
      launch_hist_batched(A(s, FP_HIST), M(FP_HIST), N(FP_HIST), ws); count(FP_HIST);
      launch_scan_batched(0, A(s, FP_SCANR), M(FP_SCANR), N(FP_SCANR), ws); count(FP_SCANR);
      launch_scan_batched(1, A(s, FP_SCANT), M(FP_SCANT), N(FP_SCANT), ws); count(FP_SCANT);
      launch_scan_batched(2, A(s, FP_SCAND), M(FP_SCAND), N(FP_SCAND), ws); count(FP_SCAND);
      launch_scatter_batched(A(s, FP_SCATTER), M(FP_SCATTER), N(FP_SCATTER), ws); count(FP_SCATTER);
    }
    if (mom_at[s]) {
      launch_moments_batched(false, A(s, FP_MOM), M(FP_MOM), N(FP_MOM), ws); count(FP_MOM);
      launch_moments_batched(true, A(s, FP_MOMFIN), M(FP_MOMFIN), N(FP_MOMFIN), ws); count(FP_MOMFIN);
    }
    cudaEventRecord(b->walk_ev[par], ws);
    walk_rec[par] = true;
  }
  cudaStreamWaitEvent(b->origin, b->walk_ev[(L - 1) & 1], 0);   // the chunk ends with every walker
  launch_advance_batched(A(L - 1, FP_ADV), M(FP_ADV), N(FP_ADV), b->origin); count(FP_ADV);
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamEndCapture(b->origin, &graph));
  cudaError_t ie = cudaGraphInstantiate(&fg.exec, graph, 0);
  cudaGraphDestroy(graph);
  BCK(ie);
  fg.launches = launches;
  return RWMI_OK;
}

rwmi_status fused_step(rwmi_batch* b, int32_t nsteps) {
  if (!b->maps) {
    const rwmi_status st = fused_build_maps(b);
    if (st != RWMI_OK) return st;
  }
  for (int32_t done_steps = 0; done_steps < nsteps; done_steps += (int32_t)b->L) {
    std::vector<int> key;
    for (rwmi_ctx* c : b->ctxs) { key.push_back(c->fcur); key.push_back(c->pcur); c->stepped = true; }
    auto it = b->fgraphs.find(key);
    if (it == b->fgraphs.end()) {
      FusedGraph fg;
      const rwmi_status st = fused_capture(b, fg);   // advances the mirrors of one chunk
      if (st != RWMI_OK) {
        if (fg.args) cudaFreeAsync(fg.args, b->origin);
        return st;
      }
      b->fgraphs[key] = fg;
      BCK(cudaGraphLaunch(fg.exec, b->origin));
      b->launches += fg.launches;
    } else {
      BCK(cudaGraphLaunch(it->second.exec, b->origin));
      b->launches += it->second.launches;
      for (rwmi_ctx* c : b->ctxs) advance_mirrors(c, b->L);
    }
  }
  return RWMI_OK;
}

}  // namespace

RWMI_API rwmi_status rwmi_batch_create(rwmi_batch** out, rwmi_ctx* const* ctxs, int32_t n) try {
  if (!out || !ctxs || n < 1) return RWMI_E_INVALID;
  *out = nullptr;
  rwmi_batch* b = new rwmi_batch();
  for (int32_t k = 0; k < n; ++k) {
    if (!ctxs[k]) { delete b; return RWMI_E_INVALID; }
    if (ctxs[k]->broken) { delete b; return RWMI_E_STATE; }
    b->ctxs.push_back(ctxs[k]);
  }
  b->L = chunk_length(ctxs[0]);
  for (rwmi_ctx* c : b->ctxs)
    if (chunk_length(c) != b->L || b->L > 64) {
      delete b;
      return RWMI_E_INVALID;   // contexts must share their sort / moment cadence
    }
  auto init = [&]() -> rwmi_status {
    BCK(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    BCK(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    BCK(cudaStreamCreateWithFlags(&b->wst, cudaStreamNonBlocking));
    BCK(cudaEventCreateWithFlags(&b->fluid_ev, cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->walk_ev[0], cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->walk_ev[1], cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->join2, cudaEventDisableTiming));
    b->join.resize(b->ctxs.size());
    for (auto& e : b->join) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return RWMI_OK;
  };
  rwmi_status st = init();
  if (st != RWMI_OK) { rwmi_batch_destroy(b); return st; }
  b->fused = fused_pays(b);   // RWMI_BATCH_AUTO: fused for small domains every context allows it
  for (rwmi_ctx* c : b->ctxs) b->fused = b->fused && fusable(c, b->ctxs[0]);
  *out = b;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return RWMI_E_OOM;
}

RWMI_API rwmi_status rwmi_batch_step(rwmi_batch* b, int32_t nsteps) try {
  if (!b || nsteps < 0) return RWMI_E_INVALID;
  if (nsteps % b->L != 0) return batch_fail(b, RWMI_E_INVALID, "rwmi_batch_step: steps must be a multiple of the chunk");
  for (rwmi_ctx* c : b->ctxs) {
    if (c->broken) return batch_fail(b, RWMI_E_STATE, "rwmi_batch_step: a context failed earlier: " + c->err);
    if (c->t % b->L != 0) return batch_fail(b, RWMI_E_STATE, "rwmi_batch_step: a context is not at a chunk boundary");
  }
  // the contexts' own queued work precedes the batch
  for (rwmi_ctx* c : b->ctxs) {
    BCK(cudaEventRecord(b->done, c->stream));
    BCK(cudaStreamWaitEvent(b->origin, b->done, 0));
  }
  if (b->fused) {
    const rwmi_status st = fused_step(b, nsteps);
    if (st != RWMI_OK) return st;
    BCK(cudaEventRecord(b->done, b->origin));
    for (rwmi_ctx* c : b->ctxs) BCK(cudaStreamWaitEvent(c->stream, b->done, 0));
    return RWMI_OK;
  }
  for (int32_t done_steps = 0; done_steps < nsteps; done_steps += (int32_t)b->L) {
    std::vector<int> key;
    for (rwmi_ctx* c : b->ctxs) { key.push_back(c->fcur); key.push_back(c->pcur); c->stepped = true; }
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      std::vector<int64_t> l0;
      for (rwmi_ctx* c : b->ctxs) l0.push_back(c->launches);
      BCK(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
      cudaEventRecord(b->fork, b->origin);
      for (size_t k = 0; k < b->ctxs.size(); ++k) {
        rwmi_ctx* c = b->ctxs[k];
        cudaStreamWaitEvent(c->stream, b->fork, 0);
        for (int64_t st = 0; st < b->L; ++st) enqueue_step(c, st == b->L - 1);
        segment_end(c);
        cudaEventRecord(b->join[k], c->stream);
        cudaStreamWaitEvent(b->origin, b->join[k], 0);
      }
      cudaGraph_t graph = nullptr;
      BCK(cudaStreamEndCapture(b->origin, &graph));
      cudaGraphExec_t exec = nullptr;
      cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      BCK(ie);
      std::vector<int64_t> dl;
      for (size_t k = 0; k < b->ctxs.size(); ++k) dl.push_back(b->ctxs[k]->launches - l0[k]);
      b->graphs[key] = std::make_pair(exec, dl);
      BCK(cudaGraphLaunch(exec, b->origin));   // mirrors advanced while capturing
    } else {
      BCK(cudaGraphLaunch(it->second.first, b->origin));
      for (size_t k = 0; k < b->ctxs.size(); ++k) {
        b->ctxs[k]->launches += it->second.second[k];
        advance_mirrors(b->ctxs[k], b->L);
      }
    }
  }
  // later work on each context's stream follows the batch
  BCK(cudaEventRecord(b->done, b->origin));
  for (rwmi_ctx* c : b->ctxs) BCK(cudaStreamWaitEvent(c->stream, b->done, 0));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return batch_fail(b, RWMI_E_OOM, std::string("rwmi_batch_step: ") + e_.what());
}

RWMI_API rwmi_status rwmi_batch_sync(rwmi_batch* b) try {
  if (!b) return RWMI_E_INVALID;
  BCK(cudaStreamSynchronize(b->origin));
  rwmi_status worst = RWMI_OK;
  for (rwmi_ctx* c : b->ctxs) {
    const rwmi_status s = rwmi_sync(c);
    if (s < 0 && (worst >= 0 || s < worst)) worst = s;
    else if (worst == RWMI_OK && s > 0) worst = s;
  }
  return worst;
} catch (const std::exception& e_) {
  return batch_fail(b, RWMI_E_OOM, std::string("rwmi_batch_sync: ") + e_.what());
}

RWMI_API void rwmi_batch_destroy(rwmi_batch* b) {
  if (!b) return;
  if (b->origin) cudaStreamSynchronize(b->origin);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.first);
  if (b->origin) {
    fused_drop_graphs(b);
    if (b->maps) cudaFreeAsync(b->maps, b->origin);
    cudaStreamSynchronize(b->origin);
  }
  for (auto e : b->join) if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->fork2) cudaEventDestroy(b->fork2);
  if (b->join2) cudaEventDestroy(b->join2);
  if (b->fluid_ev) cudaEventDestroy(b->fluid_ev);
  if (b->walk_ev[0]) cudaEventDestroy(b->walk_ev[0]);
  if (b->walk_ev[1]) cudaEventDestroy(b->walk_ev[1]);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->wst) cudaStreamDestroy(b->wst);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

RWMI_API const char* rwmi_batch_last_error(const rwmi_batch* b) { return b ? b->err.c_str() : "null batch"; }

RWMI_API rwmi_status rwmi_batch_set_mode(rwmi_batch* b, int32_t mode) try {
  if (!b || mode < RWMI_BATCH_AUTO || mode > RWMI_BATCH_FUSED) return RWMI_E_INVALID;
  bool can = true;
  for (rwmi_ctx* c : b->ctxs) can = can && fusable(c, b->ctxs[0]);
  if (mode == RWMI_BATCH_FUSED && !can)
    return batch_fail(b, RWMI_E_INVALID, "rwmi_batch_set_mode: fused execution needs partially saturated cells, "
                                         "prescribed particles and one velocity set, storage and cadence");
  b->mode = mode;
  b->fused = mode == RWMI_BATCH_FUSED || (mode == RWMI_BATCH_AUTO && can && fused_pays(b));
  return RWMI_OK;
} catch (const std::exception& e_) {
  return batch_fail(b, RWMI_E_OOM, std::string("rwmi_batch_set_mode: ") + e_.what());
}

RWMI_API rwmi_status rwmi_batch_get_tiles(const rwmi_batch* b, rwmi_batch_tiles* out) {
  if (!b || !out) return RWMI_E_INVALID;
  *out = b->tiles;
  return RWMI_OK;
}

RWMI_API rwmi_status rwmi_batch_set_tiles(rwmi_batch* b, const rwmi_batch_tiles* t) try {
  if (!b || !t) return RWMI_E_INVALID;
  if ((t->lbm_block != 64 && t->lbm_block != 128 && t->lbm_block != 256) || t->walker_chunks_per_block < 1 ||
      t->walker_chunks_per_block > 64 || t->resolve_walkers_per_block < 256 || t->raster_bricks_per_block < 1)
    return batch_fail(b, RWMI_E_INVALID, "rwmi_batch_set_tiles: out of range");
  BCK(cudaStreamSynchronize(b->origin));
  b->tiles = *t;
  fused_drop_graphs(b);
  if (b->maps) cudaFreeAsync(b->maps, b->origin);
  b->maps = nullptr;
  return RWMI_OK;
} catch (const std::exception& e_) {
  return batch_fail(b, RWMI_E_OOM, std::string("rwmi_batch_set_tiles: ") + e_.what());
}

// Coordinate search over the fused work split: each candidate value of each tile parameter, the
// others held, is timed over `steps` steps (CUDA events on the batch stream, after one untimed
// chunk that captures its graph); the fastest value is kept before the next parameter.
RWMI_API rwmi_status rwmi_batch_autotune(rwmi_batch* b, int32_t steps, rwmi_batch_tiles* chosen) try {
  if (!b || steps <= 0 || steps % b->L != 0) return RWMI_E_INVALID;
  if (!b->fused) return batch_fail(b, RWMI_E_STATE, "rwmi_batch_autotune: the batch is not fused");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  rwmi_status st = RWMI_OK;
  auto timed = [&](const rwmi_batch_tiles& t, float* ms) -> rwmi_status {
    rwmi_status s = rwmi_batch_set_tiles(b, &t);
    if (s == RWMI_OK) s = rwmi_batch_step(b, (int32_t)b->L);
    if (s != RWMI_OK) return s;
    cudaEventRecord(e0, b->origin);
    s = rwmi_batch_step(b, steps);
    if (s != RWMI_OK) return s;
    cudaEventRecord(e1, b->origin);
    if (cudaEventSynchronize(e1) != cudaSuccess) return batch_fail(b, RWMI_E_CUDA, "rwmi_batch_autotune: timing");
    cudaEventElapsedTime(ms, e0, e1);
    return RWMI_OK;
  };
  rwmi_batch_tiles best = b->tiles;
  float best_ms = 0.0f;
  st = timed(best, &best_ms);
  const int lbm_v[] = {64, 128, 256}, chunk_v[] = {1, 2, 4, 8}, res_v[] = {2048, 8192, 32768},
            brk_v[] = {16, 64, 256};
  for (int param = 0; param < 4 && st == RWMI_OK; ++param) {
    const int* vals = param == 0 ? lbm_v : param == 1 ? chunk_v : param == 2 ? res_v : brk_v;
    const int nv = param == 1 ? 4 : 3;
    for (int k = 0; k < nv && st == RWMI_OK; ++k) {
      rwmi_batch_tiles t = best;
      int* field = param == 0 ? &t.lbm_block : param == 1 ? &t.walker_chunks_per_block
                 : param == 2 ? &t.resolve_walkers_per_block : &t.raster_bricks_per_block;
      if (*field == vals[k]) continue;
      *field = vals[k];
      float ms = 0.0f;
      st = timed(t, &ms);
      if (st == RWMI_OK && ms < best_ms) { best_ms = ms; best = t; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RWMI_OK) return st;
  st = rwmi_batch_set_tiles(b, &best);
  if (st == RWMI_OK && chosen) *chosen = best;
  return st;
} catch (const std::exception& e_) {
  return batch_fail(b, RWMI_E_OOM, std::string("rwmi_batch_autotune: ") + e_.what());
}

RWMI_API int64_t rwmi_batch_launch_count(const rwmi_batch* b) { return b ? b->launches : 0; }

RWMI_API const char* rwmi_last_error(const rwmi_ctx* c) { return c ? c->err.c_str() : noalloc_last_error(); }

RWMI_API int64_t rwmi_launch_count(const rwmi_ctx* c) { return c ? c->launches : 0; }

RWMI_API int64_t rwmi_inject_alloc_failure(int64_t after) {
  const int64_t now = g_alloc_count.load();
  g_fail_at.store(after < 0 ? -1 : now + after);
  return now;
}

RWMI_API int64_t rwmi_alloc_count(void) { return g_alloc_count.load(); }

RWMI_API int32_t rwmi_inject_wait_timeout(int32_t launches) { return tma_inject_stalls(launches); }

RWMI_API void rwmi_destroy(rwmi_ctx* c) {
  if (!c) return;
  // At process teardown the CUDA runtime may already be gone: then only host memory is freed.
  if (c->stream && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return;
  }
  drop_graphs(c);
  for (int k = 0; k < 2; ++k) {
    dfree(c, c->f[k]); dfree(c, c->acc[k]); dfree(c, c->bword[k]); dfree(c, c->bcand[k]); dfree(c, c->rlist[k]);
    dfree(c, c->pose[k]); dfree(c, c->sp[k]); dfree(c, c->cworld[k]); dfree(c, c->pos[k]); dfree(c, c->x0[k]);
  }
  dfree(c, c->wlist); dfree(c, c->wlist_n);
  dfree(c, c->u[0]); dfree(c, c->u[1]); dfree(c, c->solid[0]); dfree(c, c->solid[1]); dfree(c, c->node[0]); dfree(c, c->node[1]); dfree(c, c->d_T); dfree(c, c->status); dfree(c, c->macc);
  dfree(c, c->series); dfree(c, c->mrow); dfree(c, c->fseries); dfree(c, c->desc); dfree(c, c->cbody); dfree(c, c->rank);
  dfree(c, c->counts); dfree(c, c->offsets); dfree(c, c->bsums); dfree(c, c->scratch); dfree(c, c->wmask[0]); dfree(c, c->wmask[1]);
  dfree(c, c->dem_d); dfree(c, c->dem_b);
  dfree(c, c->ibl.base); dfree(c, c->ibl.word); dfree(c, c->ibl.cell); dfree(c, c->ibl.meta); dfree(c, c->ibl.q); dfree(c, c->ibl.g); dfree(c, c->ibl.ocell); dfree(c, c->ibl.count);
  cudaStreamSynchronize(c->stream);   // the frees have returned the memory when this returns
  for (int k = 0; k < 2 * RWMI_NPHASE; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  for (cudaEvent_t e : {c->fork_ev, c->join_ev, c->fluid_ev, c->walk_ev[0], c->walk_ev[1]})
    if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->wst) cudaStreamDestroy(c->wst);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
