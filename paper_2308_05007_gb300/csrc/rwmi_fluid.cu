// rwmi_fluid.cu -- particle poses and brick lists, metaball rasteriser, fluid set-up and
// read-back (the LBM kernel itself is in rwmi_lbm.cu).
//
// Kernels (one timestep t):
//   pose_bin_kernel   particle pose at a time (prescribed motion, or read from the free DEM's
//                     state), world control points, brick candidate lists, body force, zeroed
//                     force/momentum accumulators
//   raster_kernel     solid sub-sample count + owner for every cell of bricks that touch a
//                     particle (Eq. 3, 4x4x4 sub-samples, binary32 decisions bit-identical to
//                     the CPU oracle's)
//   node_kernel       with the paper's coupling: solid/fluid node classes of the flagged bricks
//                     and the refilling of nodes uncovered since the previous step (Eq. 27)
#include "rwmi_lattice.cuh"

namespace rwmi {

void lattice_table(int q, int32_t* e, double* w) {
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) e[3 * i + a] = q == 15 ? Lat<15>::e(i, a) : Lat<19>::e(i, a);
    const int e2 = q == 15 ? Lat<15>::e2(i) : Lat<19>::e2(i);
    w[i] = q == 15 ? (e2 == 0 ? 2.0 / 9.0 : e2 == 1 ? 1.0 / 9.0 : 1.0 / 72.0)
                   : (e2 == 0 ? 1.0 / 3.0 : e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
}

// ------------------------------------------------------------------------------------------
// Prescribed particle motion and brick candidate lists
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double wrap_d(double x, double n, int wall) {
  return wall ? x : __dsub_rn(x, __dmul_rn(n, floor(__ddiv_rn(x, n))));
}

struct PoseArgs {
  Geom g;
  ParticleSet ps;
  BrickSet bs;
  const int64_t* d_T;
  int t_offset, zero_acc;
  double F0x, F0y, F0z, fper;
  double* acc;
  int q;          // lattice (15 or 19) and Guo factor 1 - 1/(2 tau) of the pair constants
  double guo0;
};

// One block per particle, blk = p of nblk = max(P, 1) blocks (block 0 also writes the body force
// of this time).
__device__ void pose_bin_body(const PoseArgs& A, int blk, int nblk) {
  const Geom g = A.g;
  const ParticleSet ps = A.ps;
  const BrickSet bs = A.bs;
  const double F0x = A.F0x, F0y = A.F0y, F0z = A.F0z, fper = A.fper;
  double* __restrict__ acc = A.acc;
  const int64_t t = *A.d_T + A.t_offset;
  if (blk == 0) {   // block-uniform: the body force of this time and the Guo pair constants
    __shared__ double s_F[3];
    if (threadIdx.x == 0) {
      const double s = fper > 0.0 ? sin(2.0 * 3.141592653589793 * (double)t / fper) : 1.0;
      s_F[0] = F0x * s;
      s_F[1] = F0y * s;
      s_F[2] = F0z * s;
      bs.sp->Fd[0] = F0x * s;
      bs.sp->Fd[1] = F0y * s;
      bs.sp->Fd[2] = F0z * s;
      bs.sp->F[0] = (float)(F0x * s);
      bs.sp->F[1] = (float)(F0y * s);
      bs.sp->F[2] = (float)(F0z * s);
    }
    __syncthreads();
    // one constant per thread (binary64 runs on a narrow pipe: a serial loop cost 4 us a step)
    const int H = (A.q - 1) / 2, j = threadIdx.x;
    if (j < 2 * H) {
      const int i = 1 + (j >> 1);
      double eF = 0.0;
      for (int a = 0; a < 3; ++a) eF += (double)(A.q == 15 ? Lat<15>::e(i, a) : Lat<19>::e(i, a)) * s_F[a];
      const double wg = (A.q == 15 ? Lat<15>::wt<double>(i) : Lat<19>::wt<double>(i)) * A.guo0;
      const double k = ((j & 1) ? 3.0 : 9.0) * wg * eF;
      guo_pairs(bs.sp)->kd[j] = k;
      guo_pairs(bs.sp)->k[j] = (float)k;
    }
  }
  if (A.zero_acc) {   // force/torque [6P] + striped mass/momentum [4 RED_SLOTS] accumulators of this time
    for (int m = blk * blockDim.x + threadIdx.x; m < 6 * ps.P + 4 * RED_SLOTS; m += nblk * blockDim.x)
      acc[m] = 0.0;
  }
  const int p = blk;
  if (p >= ps.P) return;
  __shared__ double sR[9], so[3], s_ow[3];   // rotation, origin, wrapped origin
  const ParticleDesc d = ps.desc[p];
  // Explicitly rounded FP64 operations in the oracle's order: the binary32 control points must
  // round identically on both sides, so no fused multiply-add here.
  if (threadIdx.x == 0) {
    const double two_pi = 6.283185307179586;
    double org[3], vel[3], spin[3];
    double wn = 0.0;
    for (int m = 0; m < 9; ++m) sR[m] = (m % 4 == 0) ? 1.0 : 0.0;
    if (ps.dem) {   // free DEM: the state's origin, velocity, spin and orientation quaternion
      const double* st = ps.dem + 13 * p;
      for (int a = 0; a < 3; ++a) { org[a] = st[a]; vel[a] = st[7 + a]; spin[a] = st[10 + a]; }
      const double w = st[3], x = st[4], y = st[5], z = st[6];
      sR[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, y), __dmul_rn(z, z))));
      sR[1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
      sR[2] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
      sR[3] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
      sR[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(z, z))));
      sR[5] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
      sR[6] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
      sR[7] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
      sR[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))));
    } else {
      double s = 0.0, cdt = 0.0;
      if (d.period > 0.0) {
        const double th = __dadd_rn(__ddiv_rn(__dmul_rn(two_pi, (double)t), d.period), d.phase);
        s = sin(th);
        cdt = cos(th) * two_pi / d.period;
      }
      for (int a = 0; a < 3; ++a) {
        org[a] = __dadd_rn(d.org[a], __dmul_rn(d.amp[a], s));
        vel[a] = d.amp[a] * cdt;
        spin[a] = d.omega[a];
      }
      // constant spin: body frame turned by |omega| t about omega / |omega| (Rodrigues)
      wn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d.omega[0], d.omega[0]), __dmul_rn(d.omega[1], d.omega[1])),
                                __dmul_rn(d.omega[2], d.omega[2])));
    }
    if (wn > 0.0) {
      const double ax[3] = {__ddiv_rn(d.omega[0], wn), __ddiv_rn(d.omega[1], wn), __ddiv_rn(d.omega[2], wn)};
      const double ang = __dmul_rn(wn, (double)t), ca = cos(ang), sa = sin(ang);
      const double K[9] = {0, -ax[2], ax[1], ax[2], 0, -ax[0], -ax[1], ax[0], 0};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          sR[3 * a + b] = __dadd_rn(__dadd_rn(a == b ? ca : 0.0, __dmul_rn(sa, K[3 * a + b])),
                                    __dmul_rn(__dmul_rn(__dsub_rn(1.0, ca), ax[a]), ax[b]));
    }
    for (int a = 0; a < 3; ++a) so[a] = org[a];
    PoseF pf;
    for (int a = 0; a < 3; ++a) {
      pf.o[a] = (float)wrap_d(org[a], (double)g.n[a], g.wall[a]);
      pf.v[a] = (float)vel[a];
      pf.w[a] = (float)spin[a];
      pf.pad[a] = 0.0f;
    }
    bs.pose[p] = pf;
    PoseD pd;
    for (int a = 0; a < 3; ++a) {
      pd.o[a] = wrap_d(org[a], (double)g.n[a], g.wall[a]);
      pd.v[a] = vel[a];
      pd.w[a] = spin[a];
      s_ow[a] = pd.o[a];
    }
    pd.pad = 0.0;
    bs.posed[p] = pd;
  }
  __syncthreads();
  for (int i = d.c0 + threadIdx.x; i < d.c1; i += blockDim.x) {
    const float4 cb = ps.cbody[i];
    const double b[3] = {cb.x, cb.y, cb.z};
    float4 cw;
    double w3[3];
    for (int a = 0; a < 3; ++a) {
      const double v = __dadd_rn(__dadd_rn(__dadd_rn(so[a], __dmul_rn(sR[3 * a], b[0])),
                                           __dmul_rn(sR[3 * a + 1], b[1])),
                                 __dmul_rn(sR[3 * a + 2], b[2]));
      w3[a] = wrap_d(v, (double)g.n[a], g.wall[a]);
    }
    cw.x = (float)w3[0]; cw.y = (float)w3[1]; cw.z = (float)w3[2]; cw.w = cb.w;
    bs.cworld[i] = cw;
  }
  // bricks within rb + walk_margin of the origin; raster-relevant within rb + 1. The wrapped
  // origin comes from thread 0 (an FP64 division per axis in every thread saturated the narrow
  // FP64 pipe).
  const double ow[3] = {s_ow[0], s_ow[1], s_ow[2]};
  // walker candidates and raster candidates coincide: the raster also writes the walkers'
  // mini-brick masks, which must cover every particle within the walker margin
  const float Rw = d.rb + ps.walk_margin, Rr = Rw;
  // Per axis, the bricks met by the interval [o - Rw, o + Rw] of the wrapped domain: one range,
  // or two when the interval crosses a periodic face (bricks need not tile a periodic axis
  // evenly, so the wrap is done on cell coordinates, not brick indices).
  int ra[3][2], rb_[3][2], nr[3];
  for (int a = 0; a < 3; ++a) {
    const double n = (double)g.n[a], lo = ow[a] - Rw, hi = ow[a] + Rw;
    const int last = g.nb[a] - 1;
    if (g.wall[a]) {
      const double l = fmax(lo, 0.0), h = fmin(hi, n);
      nr[a] = l <= h ? 1 : 0;
      ra[a][0] = min((int)floor(l / BRICK), last);
      rb_[a][0] = min((int)floor(h / BRICK), last);
    } else if (hi - lo >= n) {
      nr[a] = 1; ra[a][0] = 0; rb_[a][0] = last;
    } else {
      const double s0 = lo - n * floor(lo / n), e0 = s0 + (hi - lo);
      if (e0 < n) {
        nr[a] = 1;
        ra[a][0] = min((int)floor(s0 / BRICK), last);
        rb_[a][0] = min((int)floor(e0 / BRICK), last);
      } else {
        ra[a][0] = min((int)floor(s0 / BRICK), last); rb_[a][0] = last;
        ra[a][1] = 0; rb_[a][1] = min((int)floor((e0 - n) / BRICK), last);
        if (rb_[a][1] >= ra[a][0] - 1) { nr[a] = 1; ra[a][0] = 0; rb_[a][0] = last; }
        else nr[a] = 2;
      }
    }
  }
  const uint32_t nbrick = (uint32_t)g.nb[0] * g.nb[1] * g.nb[2];
  for (int combo = 0; combo < 8; ++combo) {
    const int sx = combo & 1, sy = (combo >> 1) & 1, sz = combo >> 2;
    if (sx >= nr[0] || sy >= nr[1] || sz >= nr[2]) continue;
    const int lo3[3] = {ra[0][sx], ra[1][sy], ra[2][sz]};
    const int cnt[3] = {rb_[0][sx] - ra[0][sx] + 1, rb_[1][sy] - ra[1][sy] + 1, rb_[2][sz] - ra[2][sz] + 1};
    const int total = cnt[0] * cnt[1] * cnt[2];
  for (int m = threadIdx.x; m < total; m += blockDim.x) {
    int bc[3] = {lo3[0] + m % cnt[0], lo3[1] + (m / cnt[0]) % cnt[1], lo3[2] + m / (cnt[0] * cnt[1])};
    float d2 = 0.0f;
    for (int a = 0; a < 3; ++a) {
      const float b0 = (float)(bc[a] * BRICK), b1 = fminf((float)((bc[a] + 1) * BRICK), (float)g.n[a]);
      const float c = 0.5f * (b0 + b1), h = 0.5f * (b1 - b0);
      float delta = (float)ow[a] - c;
      if (!g.wall[a]) {
        const float na = (float)g.n[a];
        delta -= na * rintf(delta / na);
      }
      const float da = fmaxf(fabsf(delta) - h, 0.0f);
      d2 += da * da;
    }
    bool app = false;   // this particle is the brick's first raster candidate: list the brick
    uint32_t b = 0;
    if (d2 <= Rw * Rw) {
      const bool rr = d2 <= Rr * Rr;
      b = ((uint32_t)bc[2] * g.nb[1] + bc[1]) * g.nb[0] + bc[0];
      const uint32_t old = atomicAdd(&bs.bword[b], 1u + (rr ? 65536u : 0u));
      const uint32_t slot = old & 0xffffu;
      if (slot < MAXC) bs.bcand[b * MAXC + slot] = (uint16_t)(p | (rr ? 0x8000 : 0));
      app = rr && (old >> 16) == 0u;
    }
    // one append per warp: every block's raster bricks go through the single list counter
    const unsigned am = __activemask();
    const unsigned bal = __ballot_sync(am, app);
    if (bal) {
      const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&bs.bword[nbrick], (uint32_t)__popc(bal));
      base = __shfl_sync(am, base, leader);
      if (app) bs.rlist[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)b;
    }
  }
  }
}

__global__ void pose_bin_kernel(const PoseArgs a) { pose_bin_body(a, blockIdx.x, gridDim.x); }
__global__ void pose_bin_batched(const PoseArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  pose_bin_body(args[m.domain], m.block, m.blocks);
}

// One row {t, F_0, T_0, F_1, T_1, ...} of the force series: the forces of the LBM update just
// done (acc), labelled with the steps completed t, read from the device counter, into slot
// (t / interval - 1) mod rows, so that a replayed graph writes the row of the step it runs.
__global__ void force_row_kernel(const double* __restrict__ acc, int P, double* __restrict__ base, int interval,
                                 int rows, const int64_t* __restrict__ d_T, int toff) {
  const int64_t t = *d_T + toff;
  double* row = base + (size_t)(((t / interval) - 1) % rows) * (1 + 6 * (size_t)P);
  for (int m = threadIdx.x; m < 6 * P; m += blockDim.x) row[1 + m] = acc[m];
  if (threadIdx.x == 0) row[0] = (double)t;
}
void launch_force_row(const double* acc, int P, double* base, int interval, int rows, const int64_t* d_T, int toff,
                      cudaStream_t st) {
  force_row_kernel<<<1, 256, 0, st>>>(acc, P, base, interval, rows, d_T, toff);
}

// Zeroes n words. A kernel rather than cudaMemsetAsync: inside the captured step a memset node
// stalled the concurrent branches of the pipelined schedule (measured: 0.14 ms per step).
struct ClearArgs {
  uint32_t* p;
  uint32_t n;
};
__device__ __forceinline__ void clear_body(const ClearArgs& a, int blk, int nblk) {
  for (uint32_t i = blk * blockDim.x + threadIdx.x; i < a.n; i += nblk * blockDim.x) a.p[i] = 0u;
}
__global__ void clear_u32_kernel(const ClearArgs a) { clear_body(a, blockIdx.x, gridDim.x); }
__global__ void clear_batched(const ClearArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  clear_body(args[m.domain], m.block, m.blocks);
}
int clear_grid(uint32_t n) {
  const uint32_t blocks = (n + 255) / 256;
  return (int)(blocks > 152 * 8 ? 152 * 8 : blocks);
}
void launch_clear_u32(uint32_t* p, uint32_t n, cudaStream_t st) {
  if (n == 0) return;
  clear_u32_kernel<<<clear_grid(n), 256, 0, st>>>(ClearArgs{p, n});
}
size_t clear_args_size() { return sizeof(ClearArgs); }
void clear_args(void* dst, uint32_t* p, uint32_t n) { *static_cast<ClearArgs*>(dst) = ClearArgs{p, n}; }
void launch_clear_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) clear_batched<<<nblocks, 256, 0, st>>>(static_cast<const ClearArgs*>(args), map);
}

static PoseArgs make_pose_args(const Geom& g, const ParticleSet& ps, BrickSet bs, const int64_t* d_T,
                               int t_offset, const double F0[3], double force_period, int zero_forces,
                               double* acc, int q, double tau) {
  PoseArgs a;
  a.g = g; a.ps = ps; a.bs = bs; a.d_T = d_T; a.t_offset = t_offset; a.zero_acc = zero_forces;
  a.F0x = F0[0]; a.F0y = F0[1]; a.F0z = F0[2]; a.fper = force_period; a.acc = acc;
  a.q = q; a.guo0 = 1.0 - 0.5 / tau;
  return a;
}
void launch_pose_bin(const Geom& g, const ParticleSet& ps, BrickSet bs, const int64_t* d_T,
                     int t_offset, const double F0[3], double force_period, int zero_forces,
                     double* acc, int q, double tau, cudaStream_t st) {
  const int blocks = ps.P > 0 ? ps.P : 1;
  pose_bin_kernel<<<blocks, 256, 0, st>>>(
      make_pose_args(g, ps, bs, d_T, t_offset, F0, force_period, zero_forces, acc, q, tau));
}
size_t pose_args_size() { return sizeof(PoseArgs); }
void pose_args(void* dst, const Geom& g, const ParticleSet& ps, BrickSet bs, const int64_t* d_T, int t_offset,
               const double F0[3], double force_period, int zero_forces, double* acc, int q, double tau) {
  *static_cast<PoseArgs*>(dst) =
      make_pose_args(g, ps, bs, d_T, t_offset, F0, force_period, zero_forces, acc, q, tau);
}
void launch_pose_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) pose_bin_batched<<<nblocks, 256, 0, st>>>(static_cast<const PoseArgs*>(args), map);
}

// ------------------------------------------------------------------------------------------
// Rasteriser: per cell, sub-samples (i + (a + 1/2)/4, ...) inside any particle (Eq. 3 >= 1).
// Interval bounds over the cell (half-diagonal 0.6495) and over its eight octants
// (half-diagonal 0.2165) settle most sub-samples; the rest are evaluated with a fast
// reciprocal and, when that lands within 4e-5 of 1, again with the exact binary32 sequence
// shared with the CPU oracle. Bounds are decided with a 1e-3 margin and the fast value with a
// 4e-5 margin, both far above binary32 rounding (~1e-6), so every decision equals the exact one.
// ------------------------------------------------------------------------------------------
struct CellBound { float fmax, fmin; };

// Displacement x - c: with mi, the minimum image on periodic axes; without, the plain difference
// (control points staged at the brick's nearest image, valid for every point of the brick).
template <bool MI>
__device__ __forceinline__ float disp(float x, float c, int a, const Geom& g) {
  return MI ? min_image_rn(x - c, (float)g.n[a], g.wall[a]) : x - c;
}

// Bounds of Eq. 3 over a ball of radius h about (x, y, z): every control point is at least
// r - h and at most r + h away. Fast reciprocal/sqrt: the 1e-3 decision margins dwarf their error.
template <bool MI>
__device__ __forceinline__ CellBound bound_at_t(const float4* cw, int c0, int c1, float x, float y, float z,
                                                float h, const Geom& g) {
  float fmax = 0.0f, fmin = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = disp<MI>(x, c.x, 0, g), dy = disp<MI>(y, c.y, 1, g), dz = disp<MI>(z, c.z, 2, g);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    const float rmin = fmaxf(r - h, 1e-15f), rmax = r + h;
    fmax += __fdividef(c.w, rmin * rmin);
    fmin += __fdividef(c.w, rmax * rmax);
  }
  CellBound b;
  b.fmax = fmax;
  b.fmin = fmin;
  return b;
}

// Upper/lower bounds over a ball of radius h1 and the upper bound over radius h2 (one pass).
struct Bound2 { float fmax1, fmin1, fmax2; };
template <bool MI>
__device__ __forceinline__ Bound2 bound_two_t(const float4* cw, int c0, int c1, float x, float y, float z,
                                              float h1, float h2, const Geom& g) {
  Bound2 b{0.0f, 0.0f, 0.0f};
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = disp<MI>(x, c.x, 0, g), dy = disp<MI>(y, c.y, 1, g), dz = disp<MI>(z, c.z, 2, g);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    const float a = fmaxf(r - h1, 1e-15f), bb = r + h1, cc = fmaxf(r - h2, 1e-15f);
    b.fmax1 += __fdividef(c.w, a * a);
    b.fmin1 += __fdividef(c.w, bb * bb);
    b.fmax2 += __fdividef(c.w, cc * cc);
  }
  return b;
}

// Sub-sample inside test: fast value from the staged control points; within 4e-5 of 1 the
// exact binary32 sequence shared with the CPU oracle decides, on the original wrapped points.
template <bool MI>
__device__ __forceinline__ bool subsample_inside_t(const float4* cw, int c0, int c1, const float4* cw_exact,
                                                   int e0, int e1, float x, float y, float z, const Geom& g) {
  float f = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = disp<MI>(x, c.x, 0, g), dy = disp<MI>(y, c.y, 1, g), dz = disp<MI>(z, c.z, 2, g);
    f += __fdividef(c.w, dx * dx + dy * dy + dz * dz);
  }
  if (fabsf(f - 1.0f) > 4e-5f) return f >= 1.0f;
  return metaball_exact(cw_exact, e0, e1, x, y, z, g) >= 1.0f;
}

// Two sub-samples of one lane that differ only in z (z and z + 1/2), in one pass over the
// staged control points: the point load, the x/y displacements and dx^2 + dy^2 are shared.
// Same fast-value tolerance and exact fallback as subsample_inside_t.
template <bool MI>
__device__ __forceinline__ void subsample_pair_t(const float4* cw, int c0, int c1, const float4* cw_exact, int e0,
                                                 int e1, float x, float y, float z, const Geom& g, bool& in_lo,
                                                 bool& in_hi) {
  const float zh = z + 0.5f;
  float flo = 0.0f, fhi = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = disp<MI>(x, c.x, 0, g), dy = disp<MI>(y, c.y, 1, g);
    const float dzl = disp<MI>(z, c.z, 2, g), dzh = disp<MI>(zh, c.z, 2, g);
    const float rxy = dx * dx + dy * dy;
    flo += __fdividef(c.w, rxy + dzl * dzl);
    fhi += __fdividef(c.w, rxy + dzh * dzh);
  }
  in_lo = fabsf(flo - 1.0f) > 4e-5f ? flo >= 1.0f : metaball_exact(cw_exact, e0, e1, x, y, z, g) >= 1.0f;
  in_hi = fabsf(fhi - 1.0f) > 4e-5f ? fhi >= 1.0f : metaball_exact(cw_exact, e0, e1, x, y, zh, g) >= 1.0f;
}

// Runtime dispatch on the (warp-uniform) minimum-image switch.
__device__ __forceinline__ CellBound bound_at(const float4* cw, int c0, int c1, float x, float y, float z,
                                              float h, const Geom& g, bool mi = true) {
  return mi ? bound_at_t<true>(cw, c0, c1, x, y, z, h, g) : bound_at_t<false>(cw, c0, c1, x, y, z, h, g);
}
__device__ __forceinline__ Bound2 bound_two(const float4* cw, int c0, int c1, float x, float y, float z,
                                            float h1, float h2, const Geom& g, bool mi) {
  return mi ? bound_two_t<true>(cw, c0, c1, x, y, z, h1, h2, g) : bound_two_t<false>(cw, c0, c1, x, y, z, h1, h2, g);
}
__device__ __forceinline__ bool subsample_inside(const float4* cw, int c0, int c1, bool mi,
                                                 const float4* cw_exact, int e0, int e1, float x, float y,
                                                 float z, const Geom& g) {
  return mi ? subsample_inside_t<true>(cw, c0, c1, cw_exact, e0, e1, x, y, z, g)
            : subsample_inside_t<false>(cw, c0, c1, cw_exact, e0, e1, x, y, z, g);
}

// Sub-sample s (bit s = a + 4 b + 16 c) of cell (i, j, k) inside the particle?
__device__ __forceinline__ bool subsample_bit(const float4* cw, int c0, int c1, bool mi, const float4* cw_exact,
                                              int e0, int e1, int i, int j, int k, int s, const Geom& g) {
  const int a = s & 3, b = (s >> 2) & 3, cc = s >> 4;
  return subsample_inside(cw, c0, c1, mi, cw_exact, e0, e1, (float)i + (0.125f + 0.25f * (float)a),
                          (float)j + (0.125f + 0.25f * (float)b), (float)k + (0.125f + 0.25f * (float)cc), g);
}

// Whole-cell mask evaluated by one thread (fallback when the shared queue is full).
__device__ uint64_t particle_mask_serial(const float4* cw, int c0, int c1, bool mi, const float4* cw_exact, int e0,
                                         int e1, int i, int j, int k, const Geom& g) {
  uint64_t m = 0ull;
  for (int s = 0; s < 64; ++s)
    if (subsample_bit(cw, c0, c1, mi, cw_exact, e0, e1, i, j, k, s, g)) m |= 1ull << s;
  return m;
}

constexpr int RW_WARPS = 8;        // warps (bricks in flight) per block
constexpr int RW_CENTERS = 192;    // control points one warp stages
constexpr int RW_CAND = 8;         // candidates one warp stages (more: the unstaged path)

struct RasterWarp {
  float4 cw[RW_CENTERS];           // control points at the brick's nearest image
  unsigned char mcls[RW_CAND][64]; // per candidate and mini-brick: class | walker bit << 2
  int p[RW_CAND], c0[RW_CAND], c1[RW_CAND], e0[RW_CAND], cls[RW_CAND];
};

// One warp per brick of the raster list (grid-stride over warps; no block barriers):
//  1. the brick's candidates and their control points (staged at the brick's nearest image) are
//     gathered by the lanes in parallel, and each candidate is classified for the whole brick;
//  2. mini-bricks (2^3 cells): raster class per candidate and the walkers' mask bit (Eq. 3 may
//     reach 1 within sqrt(3) + the walker step margin);
//  3. 16 rounds of 32 cells: each lane bounds Eq. 3 over its cell (outside / inside / straddling);
//     the warp then evaluates every straddling (cell, candidate) pair together, 32 sub-samples per
//     ballot, and the cell's lane folds the 64-bit mask in: count = popcount(OR of masks), owner =
//     the candidate with most sub-samples, lowest index on ties.
// All decisions use bounds with a 1e-3 margin and, within 4e-5 of f = 1, the exact binary32
// sequence shared with the CPU oracle, so counts and owners equal the oracle's bit for bit.
// With cells = 0 a launch stops after step 2: the IBB coupling reads node classes, not counts,
// and needs only the walkers' masks each step.
struct RasterArgs {
  Geom g;
  ParticleSet ps;
  BrickSet bs;
  uint16_t* solid;
  unsigned long long* status;
  int cells;
};

__device__ __forceinline__ void raster_body(const RasterArgs& A) {
  const Geom g = A.g;
  const ParticleSet ps = A.ps;
  const BrickSet bs = A.bs;
  uint16_t* __restrict__ solid = A.solid;
  unsigned long long* __restrict__ status = A.status;
  __shared__ RasterWarp s_rw[RW_WARPS];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  RasterWarp& W = s_rw[wib];
  const uint32_t nbrick = (uint32_t)g.nb[0] * g.nb[1] * g.nb[2];
  const uint32_t nlist = bs.bword[nbrick];
  unsigned long long queued = 0;
  // bricks are taken from a shared counter (bword[nbrick + 1], zero after the brick pass), one
  // per warp at a time: their cost ranges from a few bound tests to ~100 straddling cells, and a
  // fixed assignment left a long tail
  uint32_t li = 0;
  if (lane == 0) li = atomicAdd(&bs.bword[nbrick + 1], 1u);
  li = __shfl_sync(full, li, 0);
  for (; li < nlist; ) {
    const uint32_t b = (uint32_t)bs.rlist[li];
    const int bi = b % g.nb[0], bj = (b / g.nb[0]) % g.nb[1], bk = b / (g.nb[0] * g.nb[1]);
    const uint32_t nc = bs.bword[b] & 0xffffu;
    const bool over = nc > MAXC;
    // 1. candidates, in parallel over lanes; offsets of their control points by a warp scan
    int p = -1, cnt = 0, g0 = 0;
    if (!over && lane < (int)nc) {
      const uint16_t cid = bs.bcand[b * MAXC + lane];
      if (cid & 0x8000) {
        p = cid & 0x7fff;
        g0 = ps.desc[p].c0;
        cnt = ps.desc[p].c1 - g0;
      }
    }
    const unsigned rel = __ballot_sync(full, p >= 0);
    const int n = __popc(rel);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += v;
    }
    const int tot = __shfl_sync(full, incl, 31);
    const bool staged = !over && n <= RW_CAND && tot <= RW_CENTERS;
    if (staged && p >= 0) {
      const int slot = __popc(rel & ((1u << lane) - 1u));
      W.p[slot] = p; W.c0[slot] = incl - cnt; W.c1[slot] = incl; W.e0[slot] = g0;
    }
    __syncwarp();
    bool mi = true;
    if (staged) {
      const float bc[3] = {(float)(bi * BRICK) + 4.0f, (float)(bj * BRICK) + 4.0f, (float)(bk * BRICK) + 4.0f};
      const float H = 6.0f + ps.walk_margin;
      bool near_half = false;
      for (int m = 0; m < n; ++m) {
        const int len = W.c1[m] - W.c0[m];
        for (int i = lane; i < len; i += 32) {
          float4 cc = bs.cworld[W.e0[m] + i];
          float* v[3] = {&cc.x, &cc.y, &cc.z};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (g.wall[a]) continue;
            const float na = (float)g.n[a];
            const float d = *v[a] - bc[a];
            if (d > 0.5f * na) *v[a] -= na; else if (d < -0.5f * na) *v[a] += na;
            if (fabsf(*v[a] - bc[a]) > 0.5f * na - H) near_half = true;
          }
          W.cw[W.c0[m] + i] = cc;
        }
      }
      mi = __any_sync(full, near_half);
      __syncwarp();
      if (lane < n) {   // brick-level class (sub-samples lie within the half-diagonal of the brick)
        const float ex0 = (float)(bi * BRICK), ex1 = fminf((float)((bi + 1) * BRICK), (float)g.n[0]);
        const float ey0 = (float)(bj * BRICK), ey1 = fminf((float)((bj + 1) * BRICK), (float)g.n[1]);
        const float ez0 = (float)(bk * BRICK), ez1 = fminf((float)((bk + 1) * BRICK), (float)g.n[2]);
        const float hx = 0.5f * (ex1 - ex0) - 0.125f, hy = 0.5f * (ey1 - ey0) - 0.125f, hz = 0.5f * (ez1 - ez0) - 0.125f;
        const CellBound bb = bound_at(W.cw, W.c0[lane], W.c1[lane], 0.5f * (ex0 + ex1), 0.5f * (ey0 + ey1),
                                      0.5f * (ez0 + ez1), sqrtf(hx * hx + hy * hy + hz * hz), g, mi);
        W.cls[lane] = bb.fmax < 0.999f ? 0 : (bb.fmin > 1.001f ? 1 : 2);
      }
      __syncwarp();
      // 2. mini-bricks: raster class and walker bit per candidate
      for (int pr = lane; pr < 64 * n; pr += 32) {
        const int mb = pr & 63, m = pr >> 6;
        const float xm = (float)(bi * BRICK + 2 * (mb & 3)) + 1.0f, ym = (float)(bj * BRICK + 2 * ((mb >> 2) & 3)) + 1.0f,
                    zm = (float)(bk * BRICK + 2 * (mb >> 4)) + 1.0f;
        int cls = W.cls[m];
        bool need;
        if (cls == 2) {
          const Bound2 b2 = bound_two(W.cw, W.c0[m], W.c1[m], xm, ym, zm, 1.5155444f, 1.7320508f + ps.walk_margin, g, mi);
          cls = b2.fmax1 < 0.999f ? 0 : (b2.fmin1 > 1.001f ? 1 : 2);
          need = b2.fmax2 >= 0.999f;
        } else if (cls == 1) {
          need = true;
        } else {
          need = bound_at(W.cw, W.c0[m], W.c1[m], xm, ym, zm, 1.7320508f + ps.walk_margin, g, mi).fmax >= 0.999f;
        }
        W.mcls[m][mb] = (unsigned char)(cls | (need ? 4 : 0));
      }
      __syncwarp();
      bool n0 = false, n1 = false;
      for (int m = 0; m < n; ++m) {
        n0 |= (W.mcls[m][lane] & 4) != 0;
        n1 |= (W.mcls[m][lane + 32] & 4) != 0;
      }
      const unsigned lo = __ballot_sync(full, n0), hi = __ballot_sync(full, n1);
      if (lane == 0) bs.wmask[b] = ((unsigned long long)hi << 32) | lo;
    } else {
      if (lane == 0) {
        bs.wmask[b] = ~0ull;   // every walker of this brick is tested
        if (over) atomicAdd(&status[ST_BRICK_OVERFLOW], 1ull);
      }
    }
    // 3. cells, 32 per round
    for (int r = 0; A.cells && r < (BRICK * BRICK * BRICK) / 32; ++r) {
      const int cl = r * 32 + lane;
      const int lx = cl & 7, ly = (cl >> 3) & 7, lz = cl >> 6;
      const int i = bi * BRICK + lx, j = bj * BRICK + ly, k = bk * BRICK + lz;
      const bool in_dom = i < g.n[0] && j < g.n[1] && k < g.n[2];
      const int mb = (lx >> 1) + 4 * (ly >> 1) + 16 * (lz >> 1);
      uint64_t any = 0ull;
      int best = 0, bestp = -1;
      unsigned pend = 0u;
      const int ncand = staged ? n : (over ? ps.P : (int)nc);
      for (int m = 0; in_dom && m < ncand; ++m) {
        int pp, cls = 2, c0, c1;
        const float4* cw;
        bool cmi = mi;
        if (staged) {
          pp = W.p[m]; cls = W.mcls[m][mb] & 3; cw = W.cw; c0 = W.c0[m]; c1 = W.c1[m];
        } else {
          if (over) pp = m;
          else {
            const uint16_t cid = bs.bcand[b * MAXC + m];
            if (!(cid & 0x8000)) continue;
            pp = cid & 0x7fff;
          }
          cw = bs.cworld; c0 = ps.desc[pp].c0; c1 = ps.desc[pp].c1; cmi = true;
        }
        if (cls == 0) continue;
        uint64_t mk;
        if (cls == 1) {
          mk = ~0ull;
        } else {
          const CellBound cb = bound_at(cw, c0, c1, (float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f, 0.649519053f, g, cmi);
          if (cb.fmax < 0.999f) continue;
          if (cb.fmin > 1.001f) {
            mk = ~0ull;
          } else if (staged) {
            pend |= 1u << m;   // the whole warp evaluates it below
            continue;
          } else {
            mk = particle_mask_serial(cw, c0, c1, true, bs.cworld, c0, c1, i, j, k, g);
          }
        }
        const int np = __popcll(mk);
        any |= mk;
        if (np > 0 && (np > best || (np == best && pp < bestp))) { best = np; bestp = pp; }
      }
      // the warp evaluates each straddling (cell, candidate) pair: 2 x 32 sub-samples
      unsigned lanes_p = __ballot_sync(full, pend != 0u);
      while (lanes_p) {
        const int src = __ffs(lanes_p) - 1;
        const unsigned pm = __shfl_sync(full, pend, src);
        const int m = __ffs(pm) - 1;
        const int scl = __shfl_sync(full, cl, src);
        const int si = bi * BRICK + (scl & 7), sj = bj * BRICK + ((scl >> 3) & 7), sk = bk * BRICK + (scl >> 6);
        const int e0 = W.e0[m], e1 = e0 + (W.c1[m] - W.c0[m]);
        bool in_lo, in_hi;
        const float sx = (float)si + 0.125f, sy = (float)sj + 0.125f, sz = (float)sk + 0.125f;
        const float ax = 0.25f * (float)(lane & 3), ay = 0.25f * (float)((lane >> 2) & 3), az = 0.25f * (float)(lane >> 4);
        if (mi)
          subsample_pair_t<true>(W.cw, W.c0[m], W.c1[m], bs.cworld, e0, e1, sx + ax, sy + ay, sz + az, g, in_lo, in_hi);
        else
          subsample_pair_t<false>(W.cw, W.c0[m], W.c1[m], bs.cworld, e0, e1, sx + ax, sy + ay, sz + az, g, in_lo, in_hi);
        const unsigned blo = __ballot_sync(full, in_lo);
        const unsigned bhi = __ballot_sync(full, in_hi);
        if (lane == src) {
          const uint64_t mk = ((uint64_t)bhi << 32) | blo;
          const int np = __popcll(mk);
          const int pp = W.p[m];
          any |= mk;
          if (np > 0 && (np > best || (np == best && pp < bestp))) { best = np; bestp = pp; }
          pend &= ~(1u << m);
        }
        ++queued;
        lanes_p = __ballot_sync(full, pend != 0u);
      }
      if (in_dom) {
        const int count = __popcll(any);
        const uint32_t cell = ((uint32_t)k * g.n[1] + j) * g.n[0] + i;
        solid[cell] = count > 0 ? (uint16_t)(count | (bestp << 7)) : (uint16_t)0;
      }
    }
    __syncwarp();
    if (lane == 0) li = atomicAdd(&bs.bword[nbrick + 1], 1u);
    li = __shfl_sync(full, li, 0);
  }
  if (lane == 0 && queued) atomicAdd(&status[ST_RASTER_QUEUED], queued);
}

__global__ void __launch_bounds__(256, 4) raster_kernel(const RasterArgs a) { raster_body(a); }
__global__ void __launch_bounds__(256, 4) raster_batched(const RasterArgs* __restrict__ args,
                                                         const BlockMap* __restrict__ map) {
  raster_body(args[map[blockIdx.x].domain]);   // warps take the domain's bricks from its counter
}

// two blocks per SM: the raster runs beside the LBM, which takes the rest of each SM (four
// blocks per SM held every register file and left the LBM to start only as they finished;
// one block per SM made the raster itself the longer branch)
int raster_grid(int nsm) { return nsm * 2; }
void launch_raster(const Geom& g, const ParticleSet& ps, BrickSet bs, uint16_t* solid,
                   unsigned long long* status, int nsm, cudaStream_t st, bool cells) {
  if (ps.P == 0) return;
  raster_kernel<<<raster_grid(nsm), RW_WARPS * 32, 0, st>>>(RasterArgs{g, ps, bs, solid, status, cells ? 1 : 0});
}
size_t raster_args_size() { return sizeof(RasterArgs); }
void raster_args(void* dst, const Geom& g, const ParticleSet& ps, BrickSet bs, uint16_t* solid,
                 unsigned long long* status) {
  *static_cast<RasterArgs*>(dst) = RasterArgs{g, ps, bs, solid, status, 1};
}
void launch_raster_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) raster_batched<<<nblocks, RW_WARPS * 32, 0, st>>>(static_cast<const RasterArgs*>(args), map);
}

// ------------------------------------------------------------------------------------------
// Initial state, checkpoint load and read-back helpers
// ------------------------------------------------------------------------------------------
template <int Q, int STORE>
__global__ void init_pop_kernel(Geom g, void* f_, double rho0_d, double ux_d, double uy_d, double uz_d,
                                float* u) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  typename S::T* f = (typename S::T*)f_;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const R rho0 = (R)rho0_d, ux = (R)ux_d, uy = (R)uy_d, uz = (R)uz_d;
  const R uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R eu = L::e(i, 0) * ux + L::e(i, 1) * uy + L::e(i, 2) * uz;
    const R dev = R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu;
    const R w = L::template wt<R>(i);
    const R v = S::shifted ? w * rho0 * dev : w * rho0 * (R(1) + dev);
    S::st(f + (size_t)i * g.ncell_pad + c, v);
  }
  reinterpret_cast<float4*>(u)[c] = make_float4((float)ux, (float)uy, (float)uz, (float)rho0);
}

template <int Q, int STORE>
__global__ void pop_f64_kernel(Geom g, const void* f_, double rho0, double* out) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  const typename S::T* f = (const typename S::T*)f_;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double v = (double)S::ld(f + (size_t)i * g.ncell_pad + c);
    out[(size_t)i * g.ncell + c] = S::shifted ? v + L::template wt<double>(i) * rho0 : v;
  }
}

template <int Q, int STORE>
__global__ void load_pop_kernel(Geom g, const double* in, double rho0, void* f_) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  typename S::T* f = (typename S::T*)f_;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double v = in[(size_t)i * g.ncell + c];
    S::st(f + (size_t)i * g.ncell_pad + c, (R)(S::shifted ? v - L::template wt<double>(i) * rho0 : v));
  }
}

template <int Q, int STORE>
__global__ void density_kernel(Geom g, const void* f_, double rho0, float* out) {
  using S = Store<STORE>;
  using R = typename S::R;
  const typename S::T* f = (const typename S::T*)f_;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  R s = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) s += S::ld(f + (size_t)i * g.ncell_pad + c);
  out[c] = (float)(S::shifted ? (R)rho0 + s : s);
}

#define RWMI_DISPATCH(q, storage, KERNEL, ...)                                   \
  do {                                                                           \
    const dim3 grid_((g.ncell + 255) / 256);                                     \
    if ((q) == 15) {                                                             \
      if ((storage) == 0) KERNEL<15, 0><<<grid_, 256, 0, st>>>(__VA_ARGS__);     \
      else if ((storage) == 1) KERNEL<15, 1><<<grid_, 256, 0, st>>>(__VA_ARGS__);\
      else if ((storage) == 2) KERNEL<15, 2><<<grid_, 256, 0, st>>>(__VA_ARGS__);\
      else KERNEL<15, 3><<<grid_, 256, 0, st>>>(__VA_ARGS__);                    \
    } else {                                                                     \
      if ((storage) == 0) KERNEL<19, 0><<<grid_, 256, 0, st>>>(__VA_ARGS__);     \
      else if ((storage) == 1) KERNEL<19, 1><<<grid_, 256, 0, st>>>(__VA_ARGS__);\
      else if ((storage) == 2) KERNEL<19, 2><<<grid_, 256, 0, st>>>(__VA_ARGS__);\
      else KERNEL<19, 3><<<grid_, 256, 0, st>>>(__VA_ARGS__);                    \
    }                                                                            \
  } while (0)

void launch_init_populations(int q, int storage, const Geom& g, void* f, double rho0,
                             const double u0[3], float* u, cudaStream_t st) {
  RWMI_DISPATCH(q, storage, init_pop_kernel, g, f, rho0, u0[0], u0[1], u0[2], u);
}
void launch_populations_f64(int q, int storage, const Geom& g, const void* f, double rho0,
                            double* out, cudaStream_t st) {
  RWMI_DISPATCH(q, storage, pop_f64_kernel, g, f, rho0, out);
}
void launch_load_populations(int q, int storage, const Geom& g, const double* in, double rho0,
                             void* f, cudaStream_t st) {
  RWMI_DISPATCH(q, storage, load_pop_kernel, g, in, rho0, f);
}
void launch_density(int q, int storage, const Geom& g, const void* f, double rho0, float* out,
                    cudaStream_t st) {
  RWMI_DISPATCH(q, storage, density_kernel, g, f, rho0, out);
}

// Is (x, y, z) inside particle [c0, c1) by Eq. 3 in the CPU oracle's binary32 sequence? A fast
// value (fast reciprocal, contraction allowed; error ~1e-6 relative) decides outside 4e-5 of 1,
// the exact sequence inside that band, so the answer always equals the exact one.
__device__ __forceinline__ bool inside_exact(const float4* __restrict__ cw, int c0, int c1, float x, float y,
                                             float z, const Geom& g) {
  float f = 0.0f;
  for (int i = c0; i < c1; ++i) {
    const float4 c = cw[i];
    const float dx = min_image_rn(x - c.x, (float)g.n[0], g.wall[0]);
    const float dy = min_image_rn(y - c.y, (float)g.n[1], g.wall[1]);
    const float dz = min_image_rn(z - c.z, (float)g.n[2], g.wall[2]);
    f += __fdividef(c.w, dx * dx + dy * dy + dz * dz);
  }
  if (fabsf(f - 1.0f) > 4e-5f) return f >= 1.0f;
  return metaball_exact(cw, c0, c1, x, y, z, g) >= 1.0f;
}

// IBB node classes (Section 2.4.3): a cell centre is solid when Eq. 3 of some particle reaches 1
// there (binary32, the CPU oracle's operation order), owned by the lowest such particle index.
// Only cells of flagged bricks can be solid. With refill, a node solid in prev and fluid now gets
// G^eq(rho0, u_new) with u_new its former particle's rigid velocity (Eq. 27).
// Brick-major: block 2 b + h takes half h (z rows 4 h .. 4 h + 3) of brick b, so that a warp's
// cells share their brick and its candidate list.
template <int Q, int STORE>
__global__ void __launch_bounds__(256) node_kernel(Geom g, ParticleSet ps, BrickSet bs, const uint16_t* __restrict__ prev,
                                                   uint16_t* __restrict__ cur, void* f_, double rho0_d, int refill) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  const uint32_t b = blockIdx.x >> 1;
  const uint32_t l = threadIdx.x + ((blockIdx.x & 1u) << 8);
  const uint32_t bi = b % (uint32_t)g.nb[0], bj = (b / (uint32_t)g.nb[0]) % (uint32_t)g.nb[1],
                 bk = b / ((uint32_t)g.nb[0] * (uint32_t)g.nb[1]);
  const uint32_t x = bi * BRICK + (l & 7u), y = bj * BRICK + ((l >> 3) & 7u), z = bk * BRICK + (l >> 6);
  if (x >= (uint32_t)g.n[0] || y >= (uint32_t)g.n[1] || z >= (uint32_t)g.n[2]) return;
  const uint32_t c = (z * (uint32_t)g.n[1] + y) * (uint32_t)g.n[0] + x;
  const uint32_t w = bs.bword[b];
  int node = 0;
  if (w >> 16) {
    const float xs = (float)x + 0.5f, ys = (float)y + 0.5f, zs = (float)z + 0.5f;
    const uint32_t nc = w & 0xffffu;
    if (nc > MAXC) {
      for (int p = 0; p < ps.P && node == 0; ++p)
        if (inside_exact(bs.cworld, ps.desc[p].c0, ps.desc[p].c1, xs, ys, zs, g)) node = p + 1;
    } else {
      int best = 0x7fffffff;
      for (uint32_t m = 0; m < nc; ++m) {
        const int p = bs.bcand[b * MAXC + m] & 0x7fff;
        if (p < best && inside_exact(bs.cworld, ps.desc[p].c0, ps.desc[p].c1, xs, ys, zs, g)) best = p;
      }
      if (best != 0x7fffffff) node = best + 1;
    }
  }
  cur[c] = (uint16_t)node;
  if (refill && node == 0 && prev[c] != 0) {
    R un[3];
    rigid_velocity<R>(g, bs.pose, bs.posed, (int)prev[c] - 1, (R)x + R(0.5), (R)y + R(0.5), (R)z + R(0.5), un);
    const R rho0 = (R)rho0_d, uu = un[0] * un[0] + un[1] * un[1] + un[2] * un[2];
    typename S::T* f = (typename S::T*)f_;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R eu = (R)L::e(i, 0) * un[0] + (R)L::e(i, 1) * un[1] + (R)L::e(i, 2) * un[2];
      const R dev = R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu;
      const R wi = L::template wt<R>(i);
      S::st(f + (size_t)i * g.ncell_pad + c, S::shifted ? wi * rho0 * dev : wi * rho0 * (R(1) + dev));
    }
  }
}

void launch_nodes(int q, int storage, const Geom& g, const ParticleSet& ps, BrickSet bs,
                  const uint16_t* prev, uint16_t* cur, void* f, double rho0, bool refill,
                  cudaStream_t st) {
  const dim3 grid_(2u * (uint32_t)g.nb[0] * (uint32_t)g.nb[1] * (uint32_t)g.nb[2]);   // two blocks per brick
  if (q == 15) {
    if (storage == 0) node_kernel<15, 0><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
    else if (storage == 1) node_kernel<15, 1><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
    else if (storage == 2) node_kernel<15, 2><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
    else node_kernel<15, 3><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
  } else {
    if (storage == 0) node_kernel<19, 0><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
    else if (storage == 1) node_kernel<19, 1><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
    else if (storage == 2) node_kernel<19, 2><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
    else node_kernel<19, 3><<<grid_, 256, 0, st>>>(g, ps, bs, prev, cur, f, rho0, refill ? 1 : 0);
  }
}

__global__ void unpack_solid_kernel(Geom g, const uint16_t* solid, const uint32_t* bword,
                                    int32_t* count, int32_t* owner) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const uint32_t z = c / g.nxy, rem = c - z * g.nxy, y = rem / g.n[0], x = rem - y * g.n[0];
  const uint32_t b = ((z >> 3) * (uint32_t)g.nb[1] + (y >> 3)) * (uint32_t)g.nb[0] + (x >> 3);
  uint16_t sw = 0;
  if (bword[b] >> 16) sw = solid[c];
  const int n = sw & 0x7f;
  count[c] = n;
  owner[c] = n ? (sw >> 7) : -1;
}

void launch_unpack_solid(const Geom& g, const uint16_t* solid, const uint32_t* bword,
                         int32_t* count, int32_t* owner, cudaStream_t st) {
  unpack_solid_kernel<<<(g.ncell + 255) / 256, 256, 0, st>>>(g, solid, bword, count, owner);
}

__global__ void velocity_aos_kernel(Geom g, const float* u, float* out) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const float4 v = reinterpret_cast<const float4*>(u)[c];
  out[3 * (size_t)c] = v.x;
  out[3 * (size_t)c + 1] = v.y;
  out[3 * (size_t)c + 2] = v.z;
}

void launch_velocity_aos(const Geom& g, const float* u, float* out, cudaStream_t st) {
  velocity_aos_kernel<<<(g.ncell + 255) / 256, 256, 0, st>>>(g, u, out);
}

}  // namespace rwmi
