// rwmi_internal.cuh -- device data layout and small device helpers of the GB300 library.
//
// HBM layout (one context):
//   populations   f[2][Q][ncell_pad]      A/B ping-pong, direction-major (SoA), each direction
//                                         plane 128-byte aligned; binary32 (optionally shifted by
//                                         w_i rho0), binary16 shifted or binary64 shifted
//   velocity      u[ncell_pad] float4     (ux, uy, uz, rho) per cell and time parity, written by the
//                                         LBM kernel with one 16-byte store, gathered by walkers
//                                         (8 loads; one 16-byte load per node costs fewer
//                                         transactions than three 4-byte planes, measured)
//   solid         solid[ncell]            uint16: sub-sample count (bits 0-6) | owner (bits 7-15),
//                                         valid only in bricks flagged for the current time
//   bricks        8x8x8-cell bricks, per time parity: bword[nbrick+2] (walker-candidate count in
//                 bits 0-15, raster-relevant count in bits 16-31; word nbrick counts rlist, word
//                 nbrick+1 is the raster's work counter), bcand[nbrick][MAXC] (uint16 particle ids, bit 15 = raster-relevant),
//                 rlist[nbrick] (bricks holding raster-relevant particles); wmask[nbrick] 64-bit
//                 masks of 2^3-cell mini-bricks where walkers must test particles
//   particles     desc[P] (trajectory), cbody[Nc] float4 (body-frame x, y, z, k),
//                 per time parity: pose[P] and cworld[Nc] float4 (world x, y, z, k; wrapped)
//   walkers       pos[2][N] float4 {x, y, z, id bits} (unwrapped), x0[2][N] float4 start
//                 positions; the second buffers are the counting-sort targets
//   sort/bin      counts[ncell], offsets[ncell] uint32, rank[N] uint32, block sums
//   walker list   2 float4 per walker {x, id}, {x_f, slot}: walkers the second pass resolves
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda.h>   // CUtensorMap (types only; the encoder is fetched through the runtime)

namespace rwmi {

constexpr int BRICK = 8;            // brick edge in cells
constexpr int MAXC = 16;            // candidate particles stored per brick
constexpr uint32_t BWORD_EXTRA = 2; // words after the per-brick words of bword
constexpr int MAX_PARTICLES = 511;  // owner field of the solid word is 9 bits
constexpr int MAX_CENTERS = 65535;
constexpr float U_BOUND = 0.1f;     // lattice speed bound assumed by the walker candidate margin
constexpr int RED_SLOTS = 256;      // mass/momentum partial sums are striped over this many slots

// Status counters (device, unsigned long long): see rwmi_counters.
enum StatusSlot {
  ST_TYPE1 = 0, ST_TYPE2, ST_TYPE3, ST_TYPE4,
  ST_BISECT_FAIL, ST_REFILL_FAIL, ST_WALL_FAIL, ST_SEED_FAIL,
  ST_NONFINITE, ST_BRICK_OVERFLOW, ST_FAST_SPEED, ST_RESOLVED, ST_RASTER_QUEUED, ST_IBB_OVERFLOW,
  ST_TMA_TIMEOUT, ST_COUNT
};

struct ParticleDesc {
  double org[3], amp[3], omega[3];
  double period, phase;
  float rb;        // bound radius: Eq. 3 stays below 1 farther than rb from the origin
  int c0, c1;      // control points c0 .. c1-1
};

struct PoseF {     // particle state at one time: wrapped origin, velocity, spin
  float o[3], v[3], w[3];
  float pad[3];
};
struct PoseD {     // the same in binary64 (read by the binary64 LBM)
  double o[3], v[3], w[3];
  double pad;
};

constexpr int GK_PAIRS = 9;   // opposite pairs of the largest lattice (D3Q19)
struct StepParams {  // per time parity
  float F[3];      // body force density at that time (binary32)
  float pad;
  double Fd[3];    // the same in binary64 (for the binary64 LBM)
  double padd;
};
// Guo source constants of the opposite pairs (i, i + H), i = 1..H, formed in binary64 from F, the
// weights and g = 1 - 1/(2 tau): k[2 (i - 1)] = 9 w_i g (e_i.F), k[2 (i - 1) + 1] = 3 w_i g (e_i.F),
// so that the update forms a pair's source terms with one multiply-add. The block follows the
// StepParams of its time in the same allocation (guo_pairs), so StepParams itself, and with it
// the code of the update kernels that read F alone, stays as it is.
struct alignas(16) GuoPairs {
  double kd[2 * GK_PAIRS];   // read as double2
  float k[2 * GK_PAIRS];     // read as float2
};
static_assert(sizeof(StepParams) % 16 == 0, "GuoPairs follows StepParams 16-byte aligned");
__host__ __device__ inline GuoPairs* guo_pairs(StepParams* sp) { return reinterpret_cast<GuoPairs*>(sp + 1); }
__host__ __device__ inline const GuoPairs* guo_pairs(const StepParams* sp) {
  return reinterpret_cast<const GuoPairs*>(sp + 1);
}

// Geometry shared by all kernels (passed by value).
struct Geom {
  int n[3];            // cells per axis
  int nb[3];           // bricks per axis
  int wall[3];         // 1: no-slip walls normal to this axis
  uint32_t nxy;        // n[0] * n[1]
  uint32_t ncell;
  uint32_t ncell_pad;  // direction-plane stride of the population and velocity arrays (> ncell:
                       // slot ncell_pad - 1 is a spare that no cell owns)
  // fast division of a flat cell index by nx and nxy: q = (umulhi(v, m) + v) >> s
  uint32_t mx, sx, mxy, sxy;
  float inv_n[3];      // 1 / n per axis (wrapping; the result is corrected to [0, n))
};

// Divisor magic for q = (umulhi(v, m) + v) >> s, exact for 0 <= v < 2^31, 1 <= d < 2^31
// (Granlund and Montgomery 1994, the "add" variant).
inline void make_divisor(uint32_t d, uint32_t& m, uint32_t& s) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  s = l;
  m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1ull);
}

__device__ __forceinline__ uint32_t fast_div(uint32_t v, uint32_t m, uint32_t s) {
  return (__umulhi(v, m) + v) >> s;
}

// ---- Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products ----
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a = c.x, b = c.z;
    const uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, b), lo_b = 0xCD9E8D57u * b;
    c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ((r >> 8) + 1/2) 2^-24 in binary32: exact, and strictly inside (0, 1), while r >> 8 < 2^23; above
// that, (r >> 8) + 1/2 needs 25 bits and rounds to an even integer (within 2^-25 of the exact U,
// up to 1 itself). The walker noise takes its radius from the exact 1 - U there.
__device__ __forceinline__ float uniform24(uint32_t r) {
  return ((float)(r >> 8) + 0.5f) * 5.9604644775390625e-08f;
}

// Minimum image on a periodic axis, binary32, fixed rounding (no contraction).
__device__ __forceinline__ float min_image_rn(float d, float n, int wall) {
  if (!wall) {
    const float h = 0.5f * n;
    if (d > h) d = __fsub_rn(d, n);
    else if (d < -h) d = __fadd_rn(d, n);
  }
  return d;
}

// Eq. 3 in binary32 with the fixed operation order that decides sub-sample counts and seeding:
// d = x - c (one +-n minimum-image correction), r2 = (dx*dx + dy*dy) + dz*dz,
// f = ((k_0 / r2_0) + k_1 / r2_1) + ... ; every operation rounded to nearest, never fused.
__device__ __forceinline__ float metaball_exact(const float4* __restrict__ cw, int c0, int c1,
                                                float x, float y, float z, const Geom& g) {
  float f = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = min_image_rn(__fsub_rn(x, c.x), (float)g.n[0], g.wall[0]);
    const float dy = min_image_rn(__fsub_rn(y, c.y), (float)g.n[1], g.wall[1]);
    const float dz = min_image_rn(__fsub_rn(z, c.z), (float)g.n[2], g.wall[2]);
    float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
    f = __fadd_rn(f, __fdiv_rn(c.w, r2));
  }
  return f;
}

// Eq. 3 and Eq. 17 for walker decisions (binary32, contraction and fast reciprocals allowed).
__device__ __forceinline__ float metaball_grad(const float4* __restrict__ cw, int c0, int c1,
                                               float x, float y, float z, const Geom& g,
                                               float* gx, float* gy, float* gz) {
  float f = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = min_image_rn(x - c.x, (float)g.n[0], g.wall[0]);
    const float dy = min_image_rn(y - c.y, (float)g.n[1], g.wall[1]);
    const float dz = min_image_rn(z - c.z, (float)g.n[2], g.wall[2]);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float inv = __frcp_rn(r2);
    const float term = c.w * inv;
    f += term;
    const float s = -2.0f * term * inv;
    ax += s * dx; ay += s * dy; az += s * dz;
  }
  if (gx) { *gx = ax; *gy = ay; *gz = az; }
  return f;
}

__device__ __forceinline__ float metaball_value(const float4* __restrict__ cw, int c0, int c1,
                                                float x, float y, float z, const Geom& g) {
  float f = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = min_image_rn(x - c.x, (float)g.n[0], g.wall[0]);
    const float dy = min_image_rn(y - c.y, (float)g.n[1], g.wall[1]);
    const float dz = min_image_rn(z - c.z, (float)g.n[2], g.wall[2]);
    f += __fdividef(c.w, dx * dx + dy * dy + dz * dz);   // ~2 ulp; walker tests need no exact rounding
  }
  return f;
}

// Wrap a coordinate into [0, n) on a periodic axis (binary32; inv_n = 1/n rounded, the result is
// corrected once on either side). Total: for every float input the result lies in [0, n), so an
// index formed from it is always in range. Where the fast quotient is off by more than one
// period (|x| beyond about 2^23 n) the exact binary32 remainder decides; a non-finite
// coordinate maps to 0 (and is counted by the walker pass as a non-finite velocity or position).
__device__ __forceinline__ float wrap_coord(float x, float n, int wall, float inv_n) {
  if (wall) return x;
  float w = x - n * floorf(x * inv_n);
  if (w >= n) w -= n;
  if (w < 0.0f) w += n;
  if (!(w >= 0.0f && w < n)) {   // rare: huge or non-finite x
    w = fmodf(x, n);
    if (w < 0.0f) w += n;
    if (!(w >= 0.0f && w < n)) w = 0.0f;
  }
  return w;
}
__device__ __forceinline__ float wrap_coord(float x, float n, int wall) {
  return wrap_coord(x, n, wall, 1.0f / n);
}

__device__ __forceinline__ int brick_of(float xw, float yw, float zw, const Geom& g) {
  int bi = min(max((int)floorf(xw) >> 3, 0), g.nb[0] - 1);
  int bj = min(max((int)floorf(yw) >> 3, 0), g.nb[1] - 1);
  int bk = min(max((int)floorf(zw) >> 3, 0), g.nb[2] - 1);
  return (bk * g.nb[1] + bj) * g.nb[0] + bi;
}

// ---- kernel launchers (defined in the .cu files) ----
struct BrickSet {
  uint64_t* wmask;    // [nbrick] per brick: bit m set when mini-brick m (2^3 cells) may need a
                      // metaball test by walkers (written by the raster of this time)
  uint32_t* bword;    // [nbrick + 1]
  uint16_t* bcand;    // [nbrick * MAXC]
  int32_t* rlist;     // [nbrick]
  PoseF* pose;        // [P]
  PoseD* posed;       // [P], stored after pose
  float4* cworld;     // [Nc]
  StepParams* sp;     // [1]
};

struct ParticleSet {
  int P, Nc;
  const ParticleDesc* desc;   // [P]
  const float4* cbody;        // [Nc]
  float walk_margin;          // candidate margin for walkers, cells
  const double* dem = nullptr;   // free-DEM state [13 P] (origin, quaternion, velocity, spin), or
                                 // nullptr for the prescribed trajectories
};

void launch_clear_u32(uint32_t* p, uint32_t n, cudaStream_t st);
// row of the force series from the force accumulators of the update just done
void launch_force_row(const double* acc, int P, double* base, int interval, int rows, const int64_t* d_T, int toff,
                      cudaStream_t st);
// q, tau: lattice and relaxation time of the Guo pair constants written beside the body force
void launch_pose_bin(const Geom& g, const ParticleSet& ps, BrickSet bs, const int64_t* d_T,
                     int t_offset, const double F0[3], double force_period, int zero_forces,
                     double* forces, int q, double tau, cudaStream_t st);
// cells = false: brick classes and walker masks only (no per-cell sub-sample counts)
void launch_raster(const Geom& g, const ParticleSet& ps, BrickSet bs, uint16_t* solid,
                   unsigned long long* status, int nsm, cudaStream_t st, bool cells = true);
// Extra inputs of the IBB coupling: node classes of this time, (u, rho) of the previous update,
// particle descriptors (control point ranges). nullptr selects the partially saturated cells.
struct IbbArgs {
  const uint16_t* nodes = nullptr;
  const float4* uprev = nullptr;
  const ParticleDesc* desc = nullptr;
  const int32_t* base = nullptr;   // per cell: index of its first link in q (ibb links)
  const uint32_t* word = nullptr;  // per cell of a flagged brick: bit 0 solid node, bit i link i
  const float* q = nullptr;        // q of every link (Eq. 25)
  const void* g = nullptr;         // G_i of every link (Eqs. 23-25), in the arithmetic type
  int cap = 0;                     // capacity of the link list
};
// The IBB link list of a context: per cell the index of its first link (or -1 - its overflow
// slot) and its node word; per link the cell, the direction | particle << 8, q and G_i (binary32
// or binary64, 8 bytes reserved). q and G hold cap list entries followed by ocap overflow slots of
// Q - 1 links each (cells whose links did not fit in the list; ocell lists them). count: list and
// overflow append counters, two time parities each.
struct IbbLinks {
  int32_t* base = nullptr;
  uint32_t* word = nullptr;
  uint32_t *cell = nullptr, *meta = nullptr;
  float* q = nullptr;
  void* g = nullptr;
  int32_t* ocell = nullptr;
  unsigned int* count = nullptr;   // [4]: list (parity 0, 1), overflow (parity 0, 1)
  int cap = 0, ocap = 0;
};
// Links of time t (node classes nodes, bricks bs), their q and G_i from the LBM input
// populations fin and the previous velocity uprev, before the LBM update of t.
void launch_ibb_links(int q, int storage, const Geom& g, BrickSet bs, const uint16_t* nodes, const IbbLinks& lk,
                      int par, const ParticleDesc* desc, const void* fin, const float* uprev, double rho0,
                      unsigned long long* status, int nsm, cudaStream_t st);
// TMA-staged form of the update (MODE 0, partially saturated cells; binary32 or binary16
// storage, nx a multiple of 16 bytes): same results bit for bit as launch_lbm's update. The
// tensor map of each population buffer is encoded once (lbm_tma_encode); false where the
// geometry or the driver does not allow it.
bool lbm_tma_supported(int q, int storage, const Geom& g);
bool lbm_tma_encode(int q, int storage, const Geom& g, const void* f, CUtensorMap* map);
size_t lbm_tma_smem(int q, int storage);
int tma_inject_stalls(int n);   // rwmi_inject_wait_timeout; returns the previous count
void launch_lbm_tma(int q, int storage, const CUtensorMap& map, const Geom& g, const void* fin, void* fout, float* u,
                    const uint16_t* solid, BrickSet bs, double tau, double rho0, unsigned long long* status, int nsm,
                    cudaStream_t st);
// fused: the update and the reduction in one pass (binary32-shifted and binary64 storage; the
// reduction steps of every run, and every step of free-DEM runs, which read the forces each
// step). Its update stores the same bits as the plain update's.
void launch_lbm(int q, int storage, bool reduce, const Geom& g, const void* fin, void* fout,
                float* u, const uint16_t* solid, BrickSet bs, double tau, double rho0,
                double* red, double* forces, unsigned long long* status, cudaStream_t st,
                int block = 256, const IbbArgs* ibb = nullptr, bool fused = false, bool update = true);

// Free DEM (Section 2.2, Eqs. 4-11) of a context: contact law, state and per-pair memory. Pair
// slots (i < j) sit at i P + j, wall slots (particle p, face 2 axis + side) at 6 p + face.
constexpr int DEM_MAX_CP = 16;   // control points per particle the DEM takes
struct DemArgs {
  int P;
  int n[3], wall[3];
  const ParticleDesc* desc;
  const float4* cbody;
  double* st;                                  // [13 P]
  const double *mass, *Ib, *Rs;                // [P], [6 P], [P]
  double* zoom;                                // [P] internal-metaball scale
  double *xi, *xm;                             // pairs [3 P P]
  unsigned char* act;                          // pairs [P P]: in contact at the last DEM step
  double *xiw, *xmw;                           // walls [18 P]
  unsigned char* actw;                         // walls [6 P]
  double *pF, *pTi, *pTj;                      // pair force on i, torques on i and j [3 P P]
  double *wF, *wT;                             // wall force and torque [18 P]
  float4* posf;                                // [P] origin in binary32 and bound radius: reach
                                               // prefilter (conservative, with a margin)
  const double* Fe;                            // fluid force and torque [6 P], or nullptr
  double kn, etan, kt, etat, mus, g[3];
  double dt;                                   // 1 / substeps
};
// substeps DEM steps: one single-block launch for up to 128 particles, else two launches per DEM
// step (contacts, then integration); returns the number of launches
int launch_dem(const DemArgs& a, int substeps, cudaStream_t st);
// the zoom factors from the sphere radii (rwmi_set_dem)
void launch_dem_init(const DemArgs& a, cudaStream_t st);
// mass properties from the metaballs at the given densities: integer sample sums (zeroed by the
// caller, [10 P]), then mass, inertia, props [10 P] (mass, centre of mass, inertia); moves the
// body frames (cbody) and the state origins to the centres of mass
void launch_dem_mass(const DemArgs& a, unsigned long long* sums, const double* density, double* mass, double* Ib,
                     double* props, float4* cbody, cudaStream_t st);
// IBB node classes at time t (bricks bs of that time) into cur; with refill, nodes solid in prev
// and fluid now get the equilibrium at their former particle's rigid velocity (Eq. 27).
void launch_nodes(int q, int storage, const Geom& g, const ParticleSet& ps, BrickSet bs,
                  const uint16_t* prev, uint16_t* cur, void* f, double rho0, bool refill,
                  cudaStream_t st);
void launch_init_populations(int q, int storage, const Geom& g, void* f, double rho0,
                             const double u0[3], float* u, cudaStream_t st);
// Time of a launch: *d_T (the step counter at the start of the current run of steps, advanced
// only between runs) plus toff, fixed when the launch is queued or captured. Kernels of several
// steps may then run concurrently without racing on the counter.
// The flagged-walker list of the two-pass walker step is split into WLIST_STRIPES parts, each
// with its own append counter (the walkers of chunk k = w / 256 append to part k mod
// WLIST_STRIPES), so the appends do not serialise on one address. A part receives at most
// ceil(chunks / WLIST_STRIPES) chunks: capacity wlist_stripe_cap(n) walkers.
constexpr int WLIST_STRIPES = 32;
inline int64_t wlist_stripe_cap(int64_t n) {
  const int64_t blocks = (n + 255) / 256;
  return (blocks + WLIST_STRIPES - 1) / WLIST_STRIPES * 256;
}
// list_n: 2 * WLIST_STRIPES counters, one set per time parity (toff_parity = t mod 2); both
// sets must be zero before the first step.
void launch_walkers(const Geom& g, const ParticleSet& ps, BrickSet bs1, float4* pos, int64_t n,
                    const float* u, const int64_t* d_T, int toff, int toff_parity, float D,
                    uint32_t k0, uint32_t k1, unsigned long long* status, float4* list,
                    unsigned int* list_n, int nsm, cudaStream_t st);
void launch_advance(int64_t* d_T, int64_t k, cudaStream_t st);
void launch_seed(const Geom& g, const ParticleSet& ps, BrickSet bs, float4* pos, float4* x0,
                 int64_t n, const double lo[3], const double hi[3], uint32_t k0, uint32_t k1,
                 unsigned long long* status, cudaStream_t st);
void launch_set_walkers(const float* pos3, float4* pos, float4* x0, int64_t n, cudaStream_t st);
void launch_histogram(const Geom& g, const float4* pos, int64_t n, uint32_t* counts,
                      uint32_t* rank, cudaStream_t st);
void launch_scan(const uint32_t* counts, uint32_t* offsets, uint32_t* block_sums, uint32_t n,
                 cudaStream_t st);
void launch_scatter(const Geom& g, const float4* pos, const float4* x0, int64_t n,
                    const uint32_t* offsets, const uint32_t* rank, float4* pos_out,
                    float4* x0_out, cudaStream_t st);
void launch_moments(const float4* pos, const float4* x0, int64_t n, double* acc, double* base,
                    int interval, int rows, const int64_t* d_T, int toff, cudaStream_t st);
void launch_unpack_solid(const Geom& g, const uint16_t* solid, const uint32_t* bword,
                         int32_t* count, int32_t* owner, cudaStream_t st);
void launch_populations_f64(int q, int storage, const Geom& g, const void* f, double rho0,
                            double* out, cudaStream_t st);
void launch_velocity_aos(const Geom& g, const float* u, float* out, cudaStream_t st);
void launch_density(int q, int storage, const Geom& g, const void* f, double rho0, float* out,
                    cudaStream_t st);
void launch_load_populations(int q, int storage, const Geom& g, const double* in, double rho0,
                             void* f, cudaStream_t st);
void launch_scatter_pos(const Geom& g, const float4* pos, int64_t n, const uint32_t* offsets,
                        const uint32_t* rank, float4* pos_out, cudaStream_t st);
size_t scan_block_sums_size(uint32_t n);
const char* noalloc_last_error();
void lattice_table(int q, int32_t* e, double* w);

// ------------------------------------------------------------------------------------------
// Batched launches: one launch runs a phase's kernel body for many contexts ("domains").
// Every block works for one domain: map[blockIdx.x] names the domain, the block's index among
// that domain's blocks and their number, so the body sees the grid a launch for that domain
// alone would have. args holds one argument record per domain (the *_args functions below write
// one with the same parameters as the matching launch_* function; *_args_size gives its
// bytes). The single-context launch_* functions run the same bodies.
// ------------------------------------------------------------------------------------------
struct BlockMap {
  int32_t domain, block, blocks, pad;
};
size_t clear_args_size();
void clear_args(void* dst, uint32_t* p, uint32_t n);
void launch_clear_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t pose_args_size();
void pose_args(void* dst, const Geom& g, const ParticleSet& ps, BrickSet bs, const int64_t* d_T, int t_offset,
               const double F0[3], double force_period, int zero_forces, double* acc, int q, double tau);
void launch_pose_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t raster_args_size();
void raster_args(void* dst, const Geom& g, const ParticleSet& ps, BrickSet bs, uint16_t* solid,
                 unsigned long long* status);
void launch_raster_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
// LBM update (mode 0), reduce-only pass (mode 1) or both in one pass (mode 2) of the partially
// saturated cells
size_t lbm_args_size(int q, int storage);
void lbm_args(void* dst, int q, int storage, const Geom& g, const void* fin, void* fout, float* u,
              const uint16_t* solid, BrickSet bs, double tau, double rho0, double* red, double* forces);
// mode 0 the update, 1 the reduce-only pass, 2 both in one pass (binary32-shifted and binary64)
void launch_lbm_batched(int q, int storage, bool walls, int mode, const void* args, const BlockMap* map,
                        int nblocks, int block, cudaStream_t st);
size_t walker_args_size();
void walker_args(void* dst, const Geom& g, const ParticleSet& ps, BrickSet bs1, float4* pos, int64_t n,
                 const float* u, const int64_t* d_T, int toff, int toff_parity, float D, uint32_t k0,
                 uint32_t k1, unsigned long long* status, float4* list, unsigned int* list_n);
void launch_walker_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
void launch_resolve_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t hist_args_size();
void hist_args(void* dst, const Geom& g, const float4* pos, int64_t n, uint32_t* counts, uint32_t* rank);
void launch_hist_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t scan_args_size();
void scan_args(void* dst, const uint32_t* counts, uint32_t* offsets, uint32_t* block_sums, uint32_t n);
uint32_t scan_tiles(uint32_t n);   // blocks of the reduce and down-sweep passes
void launch_scan_batched(int pass, const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t scatter_args_size();
void scatter_args(void* dst, const Geom& g, const float4* pos, const float4* x0, int64_t n,
                  const uint32_t* offsets, const uint32_t* rank, float4* pos_out, float4* x0_out);
void launch_scatter_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t moments_args_size();
void moments_args(void* dst, const float4* pos, const float4* x0, int64_t n, double* acc, double* base,
                  int interval, int rows, const int64_t* d_T, int toff);
void launch_moments_batched(bool finalize, const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
size_t advance_args_size();
void advance_args(void* dst, int64_t* d_T, int64_t k);
void launch_advance_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st);
// grids a single-context launch of these phases uses (the batched launch gives each domain the same)
int walker_grid(int64_t n, int nsm);
int resolve_grid(int nsm);
int raster_grid(int nsm);
int clear_grid(uint32_t n);
int moments_grid(int64_t n);

}  // namespace rwmi
