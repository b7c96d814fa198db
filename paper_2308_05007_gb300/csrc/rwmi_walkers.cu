// rwmi_walkers.cu -- random-walk advance of solute walkers (Eq. 2, Section 2.4), seeding,
// counting sort by cell (the histogram is the concentration of Eq. 16) and FP64 moments.
#include <cstdio>
#include <mutex>

#include "rwmi.h"
#include "rwmi_internal.cuh"

namespace rwmi {

// ------------------------------------------------------------------------------------------
// Section 2.4.1: velocity at the walker by trilinear interpolation of the node values (cell
// centres). Periodic axes wrap; on a walled axis the wall plane carries u = 0 and the half cell
// between wall and first node interpolates linearly to it (the wall corner gets weight 0).
// ------------------------------------------------------------------------------------------
// xw: the coordinate wrapped into [0, n) on a periodic axis (unwrapped on a walled axis).
__device__ __forceinline__ void axis_weights(float xw, int n, int wall, int& i0, int& i1, float& w0,
                                             float& w1) {
  if (!wall) {
    const float s = xw - 0.5f;
    const float fl = floorf(s);
    w1 = s - fl;
    w0 = 1.0f - w1;
    int i = (int)fl;          // -1 .. n-1
    if (i < 0) i += n;
    i0 = i;
    i1 = i + 1 == n ? 0 : i + 1;
    return;
  }
  const float nf = (float)n;
  const float x = fminf(fmaxf(xw, 0.0f), nf);
  if (x < 0.5f) {
    i0 = 0; i1 = 0; w0 = 0.0f; w1 = 2.0f * x;                 // wall (0) .. node 0
  } else if (x >= nf - 0.5f) {
    i0 = n - 1; i1 = n - 1; w0 = 1.0f - 2.0f * (x - (nf - 0.5f)); w1 = 0.0f;   // node n-1 .. wall
  } else {
    const float s = x - 0.5f;
    const float fl = floorf(s);
    i0 = (int)fl;
    i1 = min(i0 + 1, n - 1);
    w1 = s - fl;
    w0 = 1.0f - w1;
  }
}

__device__ __forceinline__ void interp_velocity(const float* __restrict__ u, const Geom& g, float x,
                                                float y, float z, float& ux, float& uy, float& uz) {
  int ix0, ix1, iy0, iy1, iz0, iz1;
  float wx0, wx1, wy0, wy1, wz0, wz1;
  axis_weights(x, g.n[0], g.wall[0], ix0, ix1, wx0, wx1);
  axis_weights(y, g.n[1], g.wall[1], iy0, iy1, wy0, wy1);
  axis_weights(z, g.n[2], g.wall[2], iz0, iz1, wz0, wz1);
  const float4* __restrict__ u4 = reinterpret_cast<const float4*>(u);
  const uint32_t r00 = ((uint32_t)iz0 * g.n[1] + iy0) * g.n[0], r01 = ((uint32_t)iz0 * g.n[1] + iy1) * g.n[0];
  const uint32_t r10 = ((uint32_t)iz1 * g.n[1] + iy0) * g.n[0], r11 = ((uint32_t)iz1 * g.n[1] + iy1) * g.n[0];
  const uint32_t cidx[8] = {r00 + ix0, r00 + ix1, r01 + ix0, r01 + ix1,
                            r10 + ix0, r10 + ix1, r11 + ix0, r11 + ix1};
  const float cw[8] = {wz0 * wy0 * wx0, wz0 * wy0 * wx1, wz0 * wy1 * wx0, wz0 * wy1 * wx1,
                       wz1 * wy0 * wx0, wz1 * wy0 * wx1, wz1 * wy1 * wx0, wz1 * wy1 * wx1};
  float4 v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = __ldg(u4 + cidx[m]);   // (u, rho) of the 8 nodes
  float ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    ax += cw[m] * v[m].x;
    ay += cw[m] * v[m].y;
    az += cw[m] * v[m].z;
  }
  ux = ax; uy = ay; uz = az;
}

// Specular reflection at no-slip wall planes. Returns false if a coordinate stayed outside.
__device__ __forceinline__ bool wall_reflect(float* x, const Geom& g) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!g.wall[a]) continue;
    const float n = (float)g.n[a];
    for (int it = 0; it < 8; ++it) {
      if (x[a] < 0.0f) x[a] = -x[a];
      else if (x[a] > n) x[a] = 2.0f * n - x[a];
      else break;
    }
    if (x[a] < 0.0f || x[a] > n) { ok = false; x[a] = x[a] < 0.0f ? 0.0f : n; }
  }
  return ok;
}

__device__ __forceinline__ bool beyond_wall(const float* x, const Geom& g) {
  for (int a = 0; a < 3; ++a)
    if (g.wall[a] && (x[a] < 0.0f || x[a] > (float)g.n[a])) return true;
  return false;
}

struct WalkCtx {
  Geom g;
  ParticleSet ps;
  BrickSet bs;
};

__device__ __forceinline__ float f_particle(const WalkCtx& c, int p, const float* x, float* gr) {
  const float xw = wrap_coord(x[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
  const float yw = wrap_coord(x[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
  const float zw = wrap_coord(x[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
  const ParticleDesc& d = c.ps.desc[p];
  if (gr) return metaball_grad(c.bs.cworld, d.c0, d.c1, xw, yw, zw, c.g, gr, gr + 1, gr + 2);
  return metaball_value(c.bs.cworld, d.c0, d.c1, xw, yw, zw, c.g);
}

// Lowest-index particle holding x (any particle; bound-radius skip), or -1.
__device__ int inside_any(const WalkCtx& c, const float* x) {
  const float xw = wrap_coord(x[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
  const float yw = wrap_coord(x[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
  const float zw = wrap_coord(x[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
  for (int p = 0; p < c.ps.P; ++p) {
    const PoseF& pp = c.bs.pose[p];
    const float dx = min_image_rn(xw - pp.o[0], (float)c.g.n[0], c.g.wall[0]);
    const float dy = min_image_rn(yw - pp.o[1], (float)c.g.n[1], c.g.wall[1]);
    const float dz = min_image_rn(zw - pp.o[2], (float)c.g.n[2], c.g.wall[2]);
    const float rb = c.ps.desc[p].rb + 1e-3f;
    if (dx * dx + dy * dy + dz * dz > rb * rb) continue;
    const ParticleDesc& d = c.ps.desc[p];
    if (metaball_value(c.bs.cworld, d.c0, d.c1, xw, yw, zw, c.g) >= 1.0f) return p;
  }
  return -1;
}

// inside_any through the candidate list of x's own brick: a particle holding x lies within its
// bound radius of x, so it is on that list (built at the same time with a larger radius). Same
// answer (lowest index), a handful of particles instead of all; all of them when the list
// overflowed.
__device__ int inside_cand(const WalkCtx& c, const float* x) {
  const float xw = wrap_coord(x[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
  const float yw = wrap_coord(x[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
  const float zw = wrap_coord(x[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
  const int b = brick_of(xw, yw, zw, c.g);
  const uint32_t nc = c.bs.bword[b] & 0xffffu;
  if (nc > MAXC) return inside_any(c, x);
  int best = -1;
  for (uint32_t m = 0; m < nc; ++m) {
    const int p = c.bs.bcand[b * MAXC + m] & 0x7fff;
    if (best >= 0 && p > best) continue;
    const PoseF& pp = c.bs.pose[p];
    const float dx = min_image_rn(xw - pp.o[0], (float)c.g.n[0], c.g.wall[0]);
    const float dy = min_image_rn(yw - pp.o[1], (float)c.g.n[1], c.g.wall[1]);
    const float dz = min_image_rn(zw - pp.o[2], (float)c.g.n[2], c.g.wall[2]);
    const float rb = c.ps.desc[p].rb + 1e-3f;
    if (dx * dx + dy * dy + dz * dz > rb * rb) continue;
    const ParticleDesc& d = c.ps.desc[p];
    if (metaball_value(c.bs.cworld, d.c0, d.c1, xw, yw, zw, c.g) >= 1.0f) best = p;
  }
  return best;
}

// Algorithm 1: bisection from outside point a (f < 1) to inside point b (f >= 1) of particle p;
// |f(mid) - 1| < 1e-3 converges; at most 200 iterations. aout: final outside end.
__device__ bool bisect(const WalkCtx& c, int p, const float* a_in, const float* b_in, float* xi, float* aout) {
  float a[3] = {a_in[0], a_in[1], a_in[2]}, b[3] = {b_in[0], b_in[1], b_in[2]};
  bool found = false;
  for (int it = 1; it <= 200; ++it) {
    float mid[3] = {0.5f * (a[0] + b[0]), 0.5f * (a[1] + b[1]), 0.5f * (a[2] + b[2])};
    const float fm = f_particle(c, p, mid, nullptr);
    if (fabsf(fm - 1.0f) < 1e-3f) {
      xi[0] = mid[0]; xi[1] = mid[1]; xi[2] = mid[2];
      found = true;
      break;
    } else if (fm < 1.0f) {
      a[0] = mid[0]; a[1] = mid[1]; a[2] = mid[2];
    } else {
      b[0] = mid[0]; b[1] = mid[1]; b[2] = mid[2];
    }
  }
  if (aout) { aout[0] = a[0]; aout[1] = a[1]; aout[2] = a[2]; }
  return found;
}

// Section 2.4.2 refill of a type-II walker (see the oracle's reading, implemented alike).
__device__ bool refill(const WalkCtx& c, int p, const float* x, uint32_t id, uint32_t t, float amp,
                       uint32_t k0, uint32_t k1, float* xnew) {
  float gr[3];
  f_particle(c, p, x, gr);
  const float gn = sqrtf(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
  float s[3] = {1.0f, 0.0f, 0.0f};
  if (gn > 0.0f && isfinite(gn)) { s[0] = -gr[0] / gn; s[1] = -gr[1] / gn; s[2] = -gr[2] / gn; }
  float xo[3];
  bool out = false;
  for (float h = 0.5f; h <= 64.0f; h *= 2.0f) {
    xo[0] = x[0] + h * s[0]; xo[1] = x[1] + h * s[1]; xo[2] = x[2] + h * s[2];
    if (f_particle(c, p, xo, nullptr) < 1.0f) { out = true; break; }
  }
  if (!out) { xnew[0] = x[0]; xnew[1] = x[1]; xnew[2] = x[2]; return false; }
  float xs[3], aend[3];
  if (!bisect(c, p, xo, x, xs, aend)) { xs[0] = aend[0]; xs[1] = aend[1]; xs[2] = aend[2]; }
  float gs[3];
  f_particle(c, p, xs, gs);
  const float gsn = sqrtf(gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]);
  const float no[3] = {-gs[0] / gsn, -gs[1] / gsn, -gs[2] / gsn};
  const uint4 r = philox(make_uint4(id, t, 1u, 0u), k0, k1);
  const float ct = 2.0f * uniform24(r.x) - 1.0f;
  const float st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
  float sp, cp;
  sincospif(2.0f * uniform24(r.y), &sp, &cp);
  const float rad = amp * cbrtf(uniform24(r.z));
  float xr[3] = {xs[0] + rad * st * cp, xs[1] + rad * st * sp, xs[2] + rad * ct};
  wall_reflect(xr, c.g);
  if (inside_cand(c, xr) >= 0) {
    const float dn = (xr[0] - xs[0]) * no[0] + (xr[1] - xs[1]) * no[1] + (xr[2] - xs[2]) * no[2];
    if (dn < 0.0f) for (int a = 0; a < 3; ++a) xr[a] -= 2.0f * dn * no[a];
    wall_reflect(xr, c.g);
    if (inside_cand(c, xr) >= 0) {
      xr[0] = aend[0]; xr[1] = aend[1]; xr[2] = aend[2];
      if (inside_cand(c, xr) >= 0) { xnew[0] = xr[0]; xnew[1] = xr[1]; xnew[2] = xr[2]; return false; }
    }
  }
  xnew[0] = xr[0]; xnew[1] = xr[1]; xnew[2] = xr[2];
  return true;
}

// Rare path of a walker step (kept out of line so the common path keeps its registers): types
// II-IV against the particles at t+1 (candidates of the walker's brick, or all particles when the
// list overflowed or the step was unusually long). Returns event bits: 1 II, 2 III, 4 IV,
// 8 Algorithm 1 failure, 16 refill failure; writes the new position to xn.
__device__ __noinline__ unsigned resolve_particles(const WalkCtx& c, const float* x, const float* xf, float xw,
                                                   float yw, float zw, int b, uint32_t nc, bool far_step,
                                                   uint32_t id, uint32_t T, float amp, uint32_t k0, uint32_t k1,
                                                   float* xn) {
  unsigned ev = 0u;
  int pin = -1, qin = -1;
  if (nc > MAXC || far_step) {
    pin = inside_cand(c, x);
    qin = inside_cand(c, xf);
  } else {
    const float xfw = wrap_coord(xf[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
    const float yfw = wrap_coord(xf[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
    const float zfw = wrap_coord(xf[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
    for (uint32_t m = 0; m < nc; ++m) {
      const int p = c.bs.bcand[b * MAXC + m] & 0x7fff;
      const ParticleDesc& d = c.ps.desc[p];
      if ((pin < 0 || p < pin) && metaball_value(c.bs.cworld, d.c0, d.c1, xw, yw, zw, c.g) >= 1.0f) pin = p;
      if ((qin < 0 || p < qin) && metaball_value(c.bs.cworld, d.c0, d.c1, xfw, yfw, zfw, c.g) >= 1.0f) qin = p;
    }
  }
  if (pin >= 0 && qin >= 0) {            // type II: Dirichlet refill
    ev |= 1u;
    if (!refill(c, pin, x, id, T, amp, k0, k1, xn)) ev |= 16u;
  } else if (pin >= 0) {                 // type III: moves out freely
    ev |= 2u;
  } else if (qin >= 0) {                 // type IV: Algorithms 1 and 2
    ev |= 4u;
    float xi[3];
    if (!bisect(c, qin, x, xf, xi, nullptr)) {
      ev |= 8u;
      xn[0] = x[0]; xn[1] = x[1]; xn[2] = x[2];
    } else {
      float gr[3];
      f_particle(c, qin, xi, gr);
      const float gn = sqrtf(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
      const float nv[3] = {gr[0] / gn, gr[1] / gn, gr[2] / gn};
      const float ti[3] = {xf[0] - xi[0], xf[1] - xi[1], xf[2] - xi[2]};
      const float tn = ti[0] * nv[0] + ti[1] * nv[1] + ti[2] * nv[2];
      float tr[3];
      for (int a = 0; a < 3; ++a) tr[a] = xi[a] + (ti[a] - 2.0f * tn * nv[a]);
      if (beyond_wall(tr, c.g) || inside_cand(c, tr) >= 0) {
        xn[0] = x[0]; xn[1] = x[1]; xn[2] = x[2];
      } else {
        xn[0] = tr[0]; xn[1] = tr[1]; xn[2] = tr[2];
      }
    }
  }
  return ev;
}

// -2 ln U of the 24-bit uniform U = (m + 1/2) 2^-24, m = r >> 8: the square of the Box-Muller
// radius. The fast logarithm (absolute error about 4e-7 near 1) serves where -2 ln U > 4.8e-4,
// so that its error moves the radius by less than 2e-5 of a step. For the top 4096 values of m
// it would dominate the radius (and U itself rounds in binary32 once m >= 2^23), so there
// ln U = log1p(-v) of the exact v = 1 - U = (2^24 - m - 1/2) 2^-24; the result is never negative.
// (The rare branch inline measured 5 us per step faster than as an out-of-line call.)
__device__ __forceinline__ float neg2_log_uniform(uint32_t r) {
  const uint32_t m = r >> 8;
  if (m < 16777216u - 4096u) return -2.0f * __logf(uniform24(r));
  const float v = ((float)(16777216u - m) - 0.5f) * 5.9604644775390625e-08f;
  return -2.0f * log1pf(-v);
}

// pass-1 grid: every block resident at once (5 blocks of 256 threads at 48 registers per SM),
// looping over the walkers -- measured faster than one block per 256 walkers, and than grids
// that leave SM room for the kernels beside it
constexpr int WALKER_BLOCKS_PER_SM = 5;

// Pass 1, one thread per walker: Eq. 2 with dt = 1 (trilinear u, Philox + Box-Muller) and the
// walls. A walker whose mini-brick may meet a particle at t+1 (or whose list overflowed, or whose
// step was unusually long) is appended to a compact list instead of being written back; pass 2
// resolves those at full SIMT width, so this kernel carries none of the rare-path code.
// The arguments of both walker passes of one step.
struct WalkerArgs {
  WalkCtx c;
  float4* pos;
  int64_t n;
  const float* u;
  const int64_t* d_T;
  int toff;
  float amp;
  uint32_t k0, k1;
  unsigned long long* status;
  float4* list;
  unsigned int* list_n;        // this step's stripe counters
  unsigned int* list_n_next;   // the next step's (cleared by the resolve pass)
  int64_t cap;
};

__device__ __forceinline__ void walker_body(const WalkCtx& c, float4* __restrict__ pos, int64_t n,
                                            const float* __restrict__ u, const int64_t* __restrict__ d_T,
                                            int toff, float amp, uint32_t k0, uint32_t k1,
                                            unsigned long long* __restrict__ status, float4* __restrict__ list,
                                            unsigned int* list_n, int64_t cap, int blk, int nblk) {
  const int64_t T = *d_T + toff;
  // grid-stride over chunks of 256 walkers (block-uniform), so that a fixed grid leaves room on
  // every SM for the kernels that run beside this one
  // the next chunk's positions are loaded while this chunk's gathers are in flight
  float4 p4_next = make_float4(0.f, 0.f, 0.f, 0.f);
  if ((int64_t)blk * 256 + threadIdx.x < n) p4_next = pos[(int64_t)blk * 256 + threadIdx.x];
  for (int64_t chunk = blk; chunk * 256 < n; chunk += nblk) {
    const int64_t w = chunk * 256 + threadIdx.x;
    const float4 p4 = p4_next;
    if (w + (int64_t)nblk * 256 < n) p4_next = pos[w + (int64_t)nblk * 256];
    bool ev_wall = false, ev_fast = false, ev_nonfinite = false, flagged = false;
    float4 ea = make_float4(0.f, 0.f, 0.f, 0.f), eb = ea;
    if (w < n) {
      const uint32_t id = __float_as_uint(p4.w);
      const float x[3] = {p4.x, p4.y, p4.z};
      const float xw = wrap_coord(x[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
      const float yw = wrap_coord(x[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
      const float zw = wrap_coord(x[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
      // brick word and mini-brick mask of x, loaded together with the velocity gathers (the mask
      // is used only when 0 < candidates <= MAXC, where the raster wrote it)
      int b = 0;
      uint32_t nc = 0u;
      unsigned long long wm = 0ull;
      if (c.ps.P > 0) {
        b = brick_of(xw, yw, zw, c.g);
        nc = c.bs.bword[b] & 0xffffu;
        wm = c.bs.wmask[b];
      }
      float ux, uy, uz;
      interp_velocity(u, c.g, xw, yw, zw, ux, uy, uz);
      const uint4 r = philox(make_uint4(id, (uint32_t)T, 0u, 0u), k0, k1);
      // Box-Muller: radii from neg2_log_uniform (accurate where U -> 1), angle with the fast
      // sin/cos (absolute error ~4e-7, far below the 2e-5 per-step tolerance);
      // angle 2 pi U = pi + theta with theta = 2 pi (U - 1/2) in (-pi, pi)
      const float rad01 = sqrtf(neg2_log_uniform(r.x));
      const float rad23 = sqrtf(neg2_log_uniform(r.z));
      float s1, c1, s3, c3;
      __sincosf(6.2831853f * (uniform24(r.y) - 0.5f), &s1, &c1);
      __sincosf(6.2831853f * (uniform24(r.w) - 0.5f), &s3, &c3);
      s1 = -s1; c1 = -c1; c3 = -c3;
      float xf[3] = {x[0] + ux + amp * (rad01 * c1), x[1] + uy + amp * (rad01 * s1),
                     x[2] + uz + amp * (rad23 * c3)};
      if (!wall_reflect(xf, c.g)) ev_wall = true;
      if (c.ps.P > 0) {
        const float step2 = (xf[0] - x[0]) * (xf[0] - x[0]) + (xf[1] - x[1]) * (xf[1] - x[1]) +
                            (xf[2] - x[2]) * (xf[2] - x[2]);
        bool need = nc > MAXC;
        if (nc > 0 && nc <= MAXC) {   // mini-brick of x: cells (2a, 2a+1) along each axis of the brick
          const int ix = min(max((int)floorf(xw), 0), c.g.n[0] - 1), iy = min(max((int)floorf(yw), 0), c.g.n[1] - 1),
                    iz = min(max((int)floorf(zw), 0), c.g.n[2] - 1);
          const int mb = ((ix & 7) >> 1) + 4 * ((iy & 7) >> 1) + 16 * ((iz & 7) >> 1);
          need = (wm >> mb) & 1ull;
        }
        ev_fast = step2 > c.ps.walk_margin * c.ps.walk_margin;
        flagged = need || ev_fast;
      }
      // a non-finite velocity or position is counted (rwmi_sync reports it) and the walker keeps
      // its position: nothing non-finite is written back, so later binning stays defined
      ev_nonfinite = !(isfinite(ux) && isfinite(uy) && isfinite(uz)) ||
                     !(isfinite(xf[0]) && isfinite(xf[1]) && isfinite(xf[2]));
      if (ev_nonfinite) {
        flagged = false;
      } else if (!flagged) {
        pos[w] = make_float4(xf[0], xf[1], xf[2], p4.w);
      } else {
        ea = make_float4(x[0], x[1], x[2], p4.w);
        eb = make_float4(xf[0], xf[1], xf[2], __uint_as_float((uint32_t)w));
      }
    }
    const unsigned full = 0xffffffffu;
    const unsigned fl = __ballot_sync(full, flagged);
    if (fl) {   // one list reservation per warp, on this chunk's stripe of the list
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(fl) - 1;
      const int stripe = (int)(chunk % WLIST_STRIPES);
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(&list_n[stripe], (unsigned)__popc(fl));
      base = __shfl_sync(full, base, leader);
      if (flagged) {
        const size_t slot = (size_t)stripe * (size_t)cap + base + __popc(fl & ((1u << lane) - 1u));
        list[2 * slot] = ea;
        list[2 * slot + 1] = eb;
      }
    }
    if (__any_sync(full, ev_wall | ev_fast | ev_nonfinite)) {
      const bool evs[3] = {ev_wall, ev_fast, ev_nonfinite};
      const int slot[3] = {ST_WALL_FAIL, ST_FAST_SPEED, ST_NONFINITE};
  #pragma unroll
      for (int m = 0; m < 3; ++m) {
        const unsigned bal = __ballot_sync(full, evs[m]);
        if (bal && (threadIdx.x & 31) == 0) atomicAdd(&status[slot[m]], (unsigned long long)__popc(bal));
      }
    }
  }
}

// Pass 2 (fixed grid, grid-stride over the list stripes taken as one sequence): types II-IV of
// the flagged walkers, written back to their slots. Block 0 clears the other parity's counters,
// which the next step's pass 1 appends to.
__device__ __forceinline__ void resolve_body(const WalkCtx& c, float4* __restrict__ pos,
                                             const float4* __restrict__ list, const unsigned int* list_n,
                                             unsigned int* list_n_next, const int64_t* d_T, int toff, float amp,
                                             uint32_t k0, uint32_t k1, unsigned long long* __restrict__ status,
                                             int64_t cap, int blk, int nblk) {
  const int64_t T = *d_T + toff;
  // the stripes as one sequence: s_pre[k] = entries in stripes before k (first warp's scan)
  __shared__ unsigned s_pre[WLIST_STRIPES + 1];
  static_assert(WLIST_STRIPES == 32, "one lane per stripe");
  if (threadIdx.x < 32) {
    const unsigned v = list_n[threadIdx.x];
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)threadIdx.x >= o) incl += y;
    }
    s_pre[threadIdx.x + 1] = incl;
    if (threadIdx.x == 0) s_pre[0] = 0u;
    if (blk == 0) {
      if (v) atomicAdd(&status[ST_RESOLVED], (unsigned long long)v);
      list_n_next[threadIdx.x] = 0u;   // the next step's counters (nobody reads them now)
    }
  }
  __syncthreads();
  const unsigned total = s_pre[WLIST_STRIPES];
  unsigned ev_all[5] = {0u, 0u, 0u, 0u, 0u};
  const unsigned stride = nblk * blockDim.x;
  for (unsigned e = blk * blockDim.x + threadIdx.x; e < total; e += stride) {
    // stripe of entry e: the last k with s_pre[k] <= e, by bisection over the power-of-two
    // stripe count (k < WLIST_STRIPES since e < total = s_pre[WLIST_STRIPES])
    static_assert((WLIST_STRIPES & (WLIST_STRIPES - 1)) == 0, "stripe count must be a power of two");
    int k = 0;
#pragma unroll
    for (int half = WLIST_STRIPES / 2; half > 0; half >>= 1)
      if (s_pre[k + half] <= e) k += half;
    const size_t slot = (size_t)k * (size_t)cap + (e - s_pre[k]);
    const float4 a = list[2 * slot], bq = list[2 * slot + 1];
    const float x[3] = {a.x, a.y, a.z}, xf[3] = {bq.x, bq.y, bq.z};
    const uint32_t id = __float_as_uint(a.w);
    const uint32_t w = __float_as_uint(bq.w);
    const float xw = wrap_coord(x[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
    const float yw = wrap_coord(x[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
    const float zw = wrap_coord(x[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
    const int b = brick_of(xw, yw, zw, c.g);
    const uint32_t nc = c.bs.bword[b] & 0xffffu;
    const float step2 = (xf[0] - x[0]) * (xf[0] - x[0]) + (xf[1] - x[1]) * (xf[1] - x[1]) +
                        (xf[2] - x[2]) * (xf[2] - x[2]);
    const bool far_step = step2 > c.ps.walk_margin * c.ps.walk_margin;
    float xn[3] = {xf[0], xf[1], xf[2]};
    // most flagged walkers meet no particle: test x and x_f against the brick's candidates inline
    // (one pass over each candidate's control points) and take the out-of-line path only on a hit
    bool hit = far_step || nc > MAXC;
    if (!hit) {
      const float xfw = wrap_coord(xf[0], (float)c.g.n[0], c.g.wall[0], c.g.inv_n[0]);
      const float yfw = wrap_coord(xf[1], (float)c.g.n[1], c.g.wall[1], c.g.inv_n[1]);
      const float zfw = wrap_coord(xf[2], (float)c.g.n[2], c.g.wall[2], c.g.inv_n[2]);
      for (uint32_t m = 0; m < nc && !hit; ++m) {
        const ParticleDesc& d = c.ps.desc[c.bs.bcand[b * MAXC + m] & 0x7fff];
        float fa = 0.0f, fb = 0.0f;
        for (int i = d.c0; i < d.c1; ++i) {
          const float4 cc = c.bs.cworld[i];
          const float ax = min_image_rn(xw - cc.x, (float)c.g.n[0], c.g.wall[0]);
          const float ay = min_image_rn(yw - cc.y, (float)c.g.n[1], c.g.wall[1]);
          const float az = min_image_rn(zw - cc.z, (float)c.g.n[2], c.g.wall[2]);
          const float bx = min_image_rn(xfw - cc.x, (float)c.g.n[0], c.g.wall[0]);
          const float by = min_image_rn(yfw - cc.y, (float)c.g.n[1], c.g.wall[1]);
          const float bz = min_image_rn(zfw - cc.z, (float)c.g.n[2], c.g.wall[2]);
          fa += __fdividef(cc.w, ax * ax + ay * ay + az * az);
          fb += __fdividef(cc.w, bx * bx + by * by + bz * bz);
        }
        // the out-of-line path repeats the test with its own rounding: a 1e-3 margin sends every
        // walker whose value is anywhere near the surface there, so the two tests never disagree
        hit = fa >= 1.0f - 1e-3f || fb >= 1.0f - 1e-3f;
      }
    }
    unsigned ev = 0u;
    if (hit) ev = resolve_particles(c, x, xf, xw, yw, zw, b, nc, far_step, id, (uint32_t)T, amp, k0, k1, xn);
    pos[w] = make_float4(xn[0], xn[1], xn[2], a.w);
    for (int m = 0; m < 5; ++m) ev_all[m] += (ev >> m) & 1u;
  }
  const int slot[5] = {ST_TYPE2, ST_TYPE3, ST_TYPE4, ST_BISECT_FAIL, ST_REFILL_FAIL};
  for (int m = 0; m < 5; ++m) {
    unsigned v = ev_all[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&status[slot[m]], (unsigned long long)v);
  }
}

__global__ void __launch_bounds__(256, 5) walker_kernel(const WalkerArgs a) {
  walker_body(a.c, a.pos, a.n, a.u, a.d_T, a.toff, a.amp, a.k0, a.k1, a.status, a.list, a.list_n, a.cap,
              blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256, 5) walker_batched(const WalkerArgs* __restrict__ args,
                                                         const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const WalkerArgs& a = args[m.domain];
  walker_body(a.c, a.pos, a.n, a.u, a.d_T, a.toff, a.amp, a.k0, a.k1, a.status, a.list, a.list_n, a.cap,
              m.block, m.blocks);
}
__global__ void __launch_bounds__(256, 8) walker_resolve_kernel(const WalkerArgs a) {
  resolve_body(a.c, a.pos, a.list, a.list_n, a.list_n_next, a.d_T, a.toff, a.amp, a.k0, a.k1, a.status, a.cap,
               blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256, 4) resolve_batched(const WalkerArgs* __restrict__ args,
                                                          const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const WalkerArgs& a = args[m.domain];
  resolve_body(a.c, a.pos, a.list, a.list_n, a.list_n_next, a.d_T, a.toff, a.amp, a.k0, a.k1, a.status, a.cap,
               m.block, m.blocks);
}

static WalkerArgs make_walker_args(const Geom& g, const ParticleSet& ps, BrickSet bs1, float4* pos, int64_t n,
                                   const float* u, const int64_t* d_T, int toff, int toff_parity, float D,
                                   uint32_t k0, uint32_t k1, unsigned long long* status, float4* list,
                                   unsigned int* list_n) {
  WalkerArgs a;
  a.c = WalkCtx{g, ps, bs1};
  a.pos = pos; a.n = n; a.u = u; a.d_T = d_T; a.toff = toff; a.amp = sqrtf(2.0f * D);
  a.k0 = k0; a.k1 = k1; a.status = status; a.list = list;
  // counters per time parity: this step appends to list_n[par], the resolve pass clears the other
  // set for the next step (no memset launch, no completion ticket)
  a.list_n = list_n + WLIST_STRIPES * (toff_parity & 1);
  a.list_n_next = list_n + WLIST_STRIPES * ((toff_parity + 1) & 1);
  a.cap = wlist_stripe_cap(n);
  return a;
}
int walker_grid(int64_t n, int nsm) {
  const int64_t blocks = (n + 255) / 256;
  return (int)(blocks < (int64_t)nsm * WALKER_BLOCKS_PER_SM ? blocks : (int64_t)nsm * WALKER_BLOCKS_PER_SM);
}
// the resolve pass is latency-bound: 8 resident blocks per SM (32 registers; the rare particle
// path spills) and two waves of them measured best (step 0.744 against 0.754 ms at 4 per SM)
int resolve_grid(int nsm) { return nsm * 16; }

void launch_walkers(const Geom& g, const ParticleSet& ps, BrickSet bs1, float4* pos, int64_t n,
                    const float* u, const int64_t* d_T, int toff, int toff_parity, float D,
                    uint32_t k0, uint32_t k1, unsigned long long* status, float4* list,
                    unsigned int* list_n, int nsm, cudaStream_t st) {
  const WalkerArgs a = make_walker_args(g, ps, bs1, pos, n, u, d_T, toff, toff_parity, D, k0, k1, status, list, list_n);
  walker_kernel<<<(unsigned)walker_grid(n, nsm), 256, 0, st>>>(a);
  walker_resolve_kernel<<<resolve_grid(nsm), 256, 0, st>>>(a);
}
size_t walker_args_size() { return sizeof(WalkerArgs); }
void walker_args(void* dst, const Geom& g, const ParticleSet& ps, BrickSet bs1, float4* pos, int64_t n,
                 const float* u, const int64_t* d_T, int toff, int toff_parity, float D, uint32_t k0,
                 uint32_t k1, unsigned long long* status, float4* list, unsigned int* list_n) {
  *static_cast<WalkerArgs*>(dst) =
      make_walker_args(g, ps, bs1, pos, n, u, d_T, toff, toff_parity, D, k0, k1, status, list, list_n);
}
void launch_walker_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) walker_batched<<<nblocks, 256, 0, st>>>(static_cast<const WalkerArgs*>(args), map);
}
void launch_resolve_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) resolve_batched<<<nblocks, 256, 0, st>>>(static_cast<const WalkerArgs*>(args), map);
}

struct AdvanceArgs {
  int64_t* d_T;
  int64_t k;
};
__global__ void advance_kernel(int64_t* d_T, int64_t k) { *d_T += k; }
void launch_advance(int64_t* d_T, int64_t k, cudaStream_t st) { advance_kernel<<<1, 1, 0, st>>>(d_T, k); }
__global__ void advance_batched(const AdvanceArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  if (threadIdx.x == 0) {
    const AdvanceArgs& a = args[map[blockIdx.x].domain];
    *a.d_T += a.k;
  }
}
size_t advance_args_size() { return sizeof(AdvanceArgs); }
void advance_args(void* dst, int64_t* d_T, int64_t k) { *static_cast<AdvanceArgs*>(dst) = AdvanceArgs{d_T, k}; }
void launch_advance_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) advance_batched<<<nblocks, 32, 0, st>>>(static_cast<const AdvanceArgs*>(args), map);
}

// ------------------------------------------------------------------------------------------
// Seeding: walker w tries Philox counters (w, a, 2, 0); point lo + U (hi - lo) in explicitly
// rounded FP64, rounded to binary32; accepted when Eq. 3 (exact binary32 sequence) stays
// below 1 for every particle -- the same decision the CPU oracle takes.
// ------------------------------------------------------------------------------------------
__global__ void seed_kernel(Geom g, ParticleSet ps, BrickSet bs, float4* pos, float4* x0, int64_t n,
                            double lo0, double lo1, double lo2, double hi0, double hi1, double hi2,
                            uint32_t k0, uint32_t k1, unsigned long long* status) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
  float x[3] = {0.0f, 0.0f, 0.0f};
  bool ok = false;
  for (int a = 0; a < 1000 && !ok; ++a) {
    const uint4 r = philox(make_uint4((uint32_t)w, (uint32_t)a, 2u, 0u), k0, k1);
    const uint32_t rr[3] = {r.x, r.y, r.z};
    for (int d = 0; d < 3; ++d) {
      const double uu = ((double)(rr[d] >> 8) + 0.5) * 5.9604644775390625e-08;
      x[d] = __double2float_rn(__dadd_rn(lo[d], __dmul_rn(uu, __dsub_rn(hi[d], lo[d]))));
    }
    ok = true;
    if (ps.P > 0) {
      const int b = brick_of(wrap_coord(x[0], (float)g.n[0], g.wall[0]),
                             wrap_coord(x[1], (float)g.n[1], g.wall[1]),
                             wrap_coord(x[2], (float)g.n[2], g.wall[2]), g);
      const uint32_t nc = bs.bword[b] & 0xffffu;
      const uint32_t m_end = nc > MAXC ? (uint32_t)ps.P : nc;
      for (uint32_t m = 0; m < m_end && ok; ++m) {
        const int p = nc > MAXC ? (int)m : (bs.bcand[b * MAXC + m] & 0x7fff);
        if (metaball_exact(bs.cworld, ps.desc[p].c0, ps.desc[p].c1, x[0], x[1], x[2], g) >= 1.0f) ok = false;
      }
    }
  }
  if (!ok) atomicAdd(&status[ST_SEED_FAIL], 1ull);
  pos[w] = make_float4(x[0], x[1], x[2], __uint_as_float((uint32_t)w));
  x0[w] = make_float4(x[0], x[1], x[2], 0.0f);
}

void launch_seed(const Geom& g, const ParticleSet& ps, BrickSet bs, float4* pos, float4* x0,
                 int64_t n, const double lo[3], const double hi[3], uint32_t k0, uint32_t k1,
                 unsigned long long* status, cudaStream_t st) {
  if (n <= 0) return;
  seed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, ps, bs, pos, x0, n, lo[0], lo[1], lo[2],
                                                           hi[0], hi[1], hi[2], k0, k1, status);
}

__global__ void set_walkers_kernel(const float* pos3, float4* pos, float4* x0, int64_t n) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const float x = pos3[3 * w], y = pos3[3 * w + 1], z = pos3[3 * w + 2];
  pos[w] = make_float4(x, y, z, __uint_as_float((uint32_t)w));
  x0[w] = make_float4(x, y, z, 0.0f);
}

void launch_set_walkers(const float* pos3, float4* pos, float4* x0, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  set_walkers_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pos3, pos, x0, n);
}

// ------------------------------------------------------------------------------------------
// Eq. 16 binning and the counting sort by cell: histogram with warp-aggregated atomics (lanes
// holding walkers of the same cell share one atomic), exclusive scan, stable-per-rank scatter.
// ------------------------------------------------------------------------------------------
// Cell of one coordinate: the floor of the unwrapped coordinate, then its residue mod n on a
// periodic axis (the exact integer wrap of Eq. 16) or clamped to [0, n-1] on a walled one. Total:
// every float input gives an index in [0, n-1]. Below 2^22 the integer quotient path is exact
// (the binary32 quotient is off by at most one period, corrected on either side); beyond it the
// floor is an integer-valued float whose exact binary32 remainder (fmodf) is the residue; NaN and
// infinities end in cell 0 (periodic) or the clamped end (walled), never outside the box.
__device__ __forceinline__ int cell_coord(float xa, int n, int wall, float inv_n) {
  const float fl = floorf(xa);
  int i;
  if (wall) {
    i = fl >= (float)n ? n - 1 : (fl > 0.0f ? (int)fl : 0);   // NaN compares false: 0
  } else if (fabsf(xa) < 4194304.0f) {
    i = (int)fl;
    i -= n * (int)floorf((float)i * inv_n);
    if (i >= n) i -= n;
    if (i < 0) i += n;
  } else {
    float r = fmodf(fl, (float)n);
    if (r < 0.0f) r += (float)n;
    i = r >= 0.0f && r < (float)n ? (int)r : 0;
  }
  return min(max(i, 0), n - 1);
}

__device__ __forceinline__ uint32_t walker_cell(const float4& p, const Geom& g) {
  const int cx = cell_coord(p.x, g.n[0], g.wall[0], g.inv_n[0]);
  const int cy = cell_coord(p.y, g.n[1], g.wall[1], g.inv_n[1]);
  const int cz = cell_coord(p.z, g.n[2], g.wall[2], g.inv_n[2]);
  return ((uint32_t)cz * g.n[1] + cy) * g.n[0] + cx;
}

struct HistArgs {
  Geom g;
  const float4* pos;
  int64_t n;
  uint32_t* counts;
  uint32_t* rank;
};
__device__ __forceinline__ void histogram_body(const Geom& g, const float4* __restrict__ pos, int64_t n,
                                               uint32_t* __restrict__ counts, uint32_t* __restrict__ rank, int blk) {
  const int64_t w = (int64_t)blk * blockDim.x + threadIdx.x;
  const bool act = w < n;
  const unsigned amask = __ballot_sync(0xffffffffu, act);
  if (!act) return;
  const uint32_t cell = walker_cell(pos[w], g);
  // Walkers are sorted by cell up to their drift since the last sort, so equal cells mostly sit
  // in runs of neighbouring lanes: each run's first lane adds the run's length and the others
  // take their rank from it (equal cells in separate runs add separately; ranks stay a
  // permutation of 0..count-1 per cell). The active lanes are 0..popc(amask)-1.
  const int lane = threadIdx.x & 31;
  const uint32_t prev = __shfl_up_sync(amask, cell, 1);
  const bool head = lane == 0 || prev != cell;
  const unsigned heads = __ballot_sync(amask, head);
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);   // lanes 0..lane
  const int first = 31 - __clz(heads & upto);                            // this lane's run head
  uint32_t base = 0;
  if (head) {
    const unsigned later = heads & ~upto;
    const int end = later ? __ffs(later) - 1 : __popc(amask);             // one past the run
    base = atomicAdd(&counts[cell], (uint32_t)(end - lane));
  }
  base = __shfl_sync(amask, base, first);
  if (rank) rank[w] = base + (uint32_t)(lane - first);
}

__global__ void histogram_kernel(Geom g, const float4* __restrict__ pos, int64_t n,
                                 uint32_t* __restrict__ counts, uint32_t* __restrict__ rank) {
  histogram_body(g, pos, n, counts, rank, blockIdx.x);
}
__global__ void hist_batched(const HistArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const HistArgs& a = args[m.domain];
  histogram_body(a.g, a.pos, a.n, a.counts, a.rank, m.block);
}
void launch_histogram(const Geom& g, const float4* pos, int64_t n, uint32_t* counts,
                      uint32_t* rank, cudaStream_t st) {
  if (n <= 0) return;
  histogram_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, pos, n, counts, rank);
}
size_t hist_args_size() { return sizeof(HistArgs); }
void hist_args(void* dst, const Geom& g, const float4* pos, int64_t n, uint32_t* counts, uint32_t* rank) {
  *static_cast<HistArgs*>(dst) = HistArgs{g, pos, n, counts, rank};
}
void launch_hist_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) hist_batched<<<nblocks, 256, 0, st>>>(static_cast<const HistArgs*>(args), map);
}

constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

size_t scan_block_sums_size(uint32_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_w[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_w[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < SCAN_THREADS / 32 ? s_w[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < SCAN_THREADS / 32) s_w[lane] = s;
  }
  __syncthreads();
  const uint32_t wbase = wid > 0 ? s_w[wid - 1] : 0u;
  if (total) *total = s_w[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return wbase + incl - v;
}

struct ScanArgs {
  const uint32_t* in;
  uint32_t n, nb;
  uint32_t* sums;
  uint32_t* out;
};
// A thread's SCAN_ITEMS consecutive words (base is a multiple of 8): two 16-byte accesses where
// the array is 16-byte aligned and the words lie inside it, else word by word (arrays handed in
// by callers of the allocation-free binning may sit at any 4-byte offset).
static_assert(SCAN_ITEMS == 8, "two uint4 per thread");
__device__ __forceinline__ void scan_load8(const uint32_t* __restrict__ in, uint32_t base, uint32_t n, uint32_t* v) {
  if (base + 8 <= n && (reinterpret_cast<uintptr_t>(in) & 15u) == 0) {
    const uint4 a = *reinterpret_cast<const uint4*>(in + base);
    const uint4 b = *reinterpret_cast<const uint4*>(in + base + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = base + k < n ? in[base + k] : 0u;
  }
}
__device__ __forceinline__ void scan_store8(uint32_t* __restrict__ out, uint32_t base, uint32_t n, const uint32_t* v) {
  if (base + 8 <= n && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
    *reinterpret_cast<uint4*>(out + base) = make_uint4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<uint4*>(out + base + 4) = make_uint4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (base + k < n) out[base + k] = v[k];
  }
}

__device__ __forceinline__ void scan_reduce_body(const uint32_t* __restrict__ in, uint32_t n,
                                                 uint32_t* __restrict__ sums, int blk) {
  const uint32_t base = blk * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS], s = 0;
  scan_load8(in, base, n, v);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) s += v[k];
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blk] = total;
}
__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ sums) {
  scan_reduce_body(in, n, sums, blockIdx.x);
}

__device__ __forceinline__ void scan_top_body(uint32_t* sums, uint32_t nb) {
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nb; base += SCAN_THREADS) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < nb ? sums[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, &total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
}
__global__ void scan_top_kernel(uint32_t* sums, uint32_t nb) { scan_top_body(sums, nb); }

__device__ __forceinline__ void scan_down_body(const uint32_t* __restrict__ in, uint32_t n,
                                               const uint32_t* __restrict__ sums, uint32_t* __restrict__ out,
                                               int blk) {
  const uint32_t base = blk * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS], s = 0;
  scan_load8(in, base, n, v);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) s += v[k];
  uint32_t run = sums[blk] + block_exclusive_scan(s, nullptr);
  uint32_t o[SCAN_ITEMS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    o[k] = run;
    run += v[k];
  }
  scan_store8(out, base, n, o);
}

__global__ void scan_down_kernel(const uint32_t* __restrict__ in, uint32_t n,
                                 const uint32_t* __restrict__ sums, uint32_t* __restrict__ out) {
  scan_down_body(in, n, sums, out, blockIdx.x);
}
// pass 0: tile sums, 1: scan of the tile sums (one block per domain), 2: down-sweep
__global__ void scan_batched(int pass, const ScanArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const ScanArgs& a = args[m.domain];
  if (pass == 0) scan_reduce_body(a.in, a.n, a.sums, m.block);
  else if (pass == 1) scan_top_body(a.sums, a.nb);
  else scan_down_body(a.in, a.n, a.sums, a.out, m.block);
}
uint32_t scan_tiles(uint32_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }
size_t scan_args_size() { return sizeof(ScanArgs); }
void scan_args(void* dst, const uint32_t* counts, uint32_t* offsets, uint32_t* block_sums, uint32_t n) {
  *static_cast<ScanArgs*>(dst) = ScanArgs{counts, n, scan_tiles(n), block_sums, offsets};
}
void launch_scan_batched(int pass, const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) scan_batched<<<nblocks, SCAN_THREADS, 0, st>>>(pass, static_cast<const ScanArgs*>(args), map);
}

void launch_scan(const uint32_t* counts, uint32_t* offsets, uint32_t* block_sums, uint32_t n,
                 cudaStream_t st) {
  const uint32_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  scan_reduce_kernel<<<nb, SCAN_THREADS, 0, st>>>(counts, n, block_sums);
  scan_top_kernel<<<1, SCAN_THREADS, 0, st>>>(block_sums, nb);
  scan_down_kernel<<<nb, SCAN_THREADS, 0, st>>>(counts, n, block_sums, offsets);
}

struct ScatterArgs {
  Geom g;
  const float4* pos;
  const float4* x0;
  int64_t n;
  const uint32_t* offsets;
  const uint32_t* rank;
  float4* pos_out;
  float4* x0_out;
};
__device__ __forceinline__ void scatter_body(const Geom& g, const float4* __restrict__ pos,
                                             const float4* __restrict__ x0, int64_t n,
                                             const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ rank,
                                             float4* __restrict__ pos_out, float4* __restrict__ x0_out, int blk) {
  const int64_t w = (int64_t)blk * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const float4 p = pos[w];
  const uint32_t dst = offsets[walker_cell(p, g)] + rank[w];
  pos_out[dst] = p;
  x0_out[dst] = x0[w];
}
__global__ void scatter_kernel(Geom g, const float4* __restrict__ pos, const float4* __restrict__ x0,
                               int64_t n, const uint32_t* __restrict__ offsets,
                               const uint32_t* __restrict__ rank, float4* __restrict__ pos_out,
                               float4* __restrict__ x0_out) {
  scatter_body(g, pos, x0, n, offsets, rank, pos_out, x0_out, blockIdx.x);
}
__global__ void scatter_batched(const ScatterArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const ScatterArgs& a = args[m.domain];
  scatter_body(a.g, a.pos, a.x0, a.n, a.offsets, a.rank, a.pos_out, a.x0_out, m.block);
}
size_t scatter_args_size() { return sizeof(ScatterArgs); }
void scatter_args(void* dst, const Geom& g, const float4* pos, const float4* x0, int64_t n,
                  const uint32_t* offsets, const uint32_t* rank, float4* pos_out, float4* x0_out) {
  *static_cast<ScatterArgs*>(dst) = ScatterArgs{g, pos, x0, n, offsets, rank, pos_out, x0_out};
}
void launch_scatter_batched(const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0) scatter_batched<<<nblocks, 256, 0, st>>>(static_cast<const ScatterArgs*>(args), map);
}

__global__ void scatter_pos_kernel(Geom g, const float4* __restrict__ pos, int64_t n,
                                   const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ rank,
                                   float4* __restrict__ pos_out) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const float4 p = pos[w];
  pos_out[offsets[walker_cell(p, g)] + rank[w]] = p;
}

void launch_scatter_pos(const Geom& g, const float4* pos, int64_t n, const uint32_t* offsets,
                        const uint32_t* rank, float4* pos_out, cudaStream_t st) {
  if (n <= 0) return;
  scatter_pos_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, pos, n, offsets, rank, pos_out);
}

void launch_scatter(const Geom& g, const float4* pos, const float4* x0, int64_t n,
                    const uint32_t* offsets, const uint32_t* rank, float4* pos_out,
                    float4* x0_out, cudaStream_t st) {
  if (n <= 0) return;
  scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, pos, x0, n, offsets, rank, pos_out, x0_out);
}

// ------------------------------------------------------------------------------------------
// FP64 walker moments: sums of d = x - x0, d^2, x, x^2 per axis (exact FP64 differences of the
// binary32 positions), then {N, mean d, var d, mean x, var x}.
// ------------------------------------------------------------------------------------------
// Float-float (double-binary32) accumulation: a value hi + lo carried exactly by error-free
// transformations (Knuth's TwoSum, FMA TwoProduct), about 48 significant bits. It replaces the
// per-walker binary64 arithmetic, which GB300's narrow FP64 pipe made the cost of the moments.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// acc += (th + tl), then renormalised
__device__ __forceinline__ void ff_acc(FF& acc, float th, float tl) {
  const FF s = ff_two_sum(acc.hi, th);
  const float e = __fadd_rn(s.lo, __fadd_rn(acc.lo, tl));
  const float hi = __fadd_rn(s.hi, e);
  acc.lo = __fsub_rn(e, __fsub_rn(hi, s.hi));
  acc.hi = hi;
}

struct MomentArgs {
  const float4* pos;
  const float4* x0;
  int64_t n;
  double* acc;
  double* base;
  int interval, rows;
  const int64_t* d_T;
  int toff;
};
__device__ __forceinline__ void moments_body(const float4* __restrict__ pos, const float4* __restrict__ x0,
                                             int64_t n, double* __restrict__ acc, int blk, int nblk) {
  FF a[12];
#pragma unroll
  for (int m = 0; m < 12; ++m) a[m] = {0.0f, 0.0f};
  for (int64_t w = (int64_t)blk * blockDim.x + threadIdx.x; w < n; w += (int64_t)nblk * blockDim.x) {
    const float4 p = pos[w], q = x0[w];
    const float xs[3] = {p.x, p.y, p.z}, x0s[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const FF d = ff_two_sum(xs[k], -x0s[k]);                 // x - x0, exact
      ff_acc(a[k], d.hi, d.lo);
      const float p2 = __fmul_rn(d.hi, d.hi);                    // d^2 = hi^2 + 2 hi lo (+ lo^2 < 2^-48 d^2)
      const float e2 = __fadd_rn(__fmaf_rn(d.hi, d.hi, -p2), __fmul_rn(2.0f, __fmul_rn(d.hi, d.lo)));
      ff_acc(a[3 + k], p2, e2);
      ff_acc(a[6 + k], xs[k], 0.0f);
      const float x2 = __fmul_rn(xs[k], xs[k]);                  // x^2 exactly as x2 + fma residue
      ff_acc(a[9 + k], x2, __fmaf_rn(xs[k], xs[k], -x2));
    }
  }
  // warp sums in float-float too; binary64 from the warp level on
#pragma unroll
  for (int m = 0; m < 12; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, a[m].hi, o), ol = __shfl_xor_sync(0xffffffffu, a[m].lo, o);
      ff_acc(a[m], oh, ol);
    }
  __shared__ double s[8][12];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane < 12) {
    float hi = a[0].hi, lo = a[0].lo;
#pragma unroll
    for (int m = 1; m < 12; ++m)
      if (lane == m) { hi = a[m].hi; lo = a[m].lo; }
    s[wid][lane] = (double)hi + (double)lo;
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s[k][threadIdx.x];
    atomicAdd(&acc[threadIdx.x], t);
  }
}
__global__ void moments_kernel(const float4* __restrict__ pos, const float4* __restrict__ x0, int64_t n,
                               double* __restrict__ acc) {
  moments_body(pos, x0, n, acc, blockIdx.x, gridDim.x);
}

// Row {t, N, mean d[3], var d[3], mean x[3], var x[3]}; clears acc for the next use. With
// interval > 0 the row is slot (t / interval - 1) mod rows of the series at base (so a replayed
// graph writes the row of the step it runs), otherwise base itself.
__device__ __forceinline__ void moments_finalize_body(double* acc, int64_t n, double* base, int interval, int rows,
                                                      const int64_t* d_T, int toff) {
  if (threadIdx.x != 0) return;
  const double N = (double)n;
  const int64_t t = *d_T + toff;
  double* out_row = base;
  if (interval > 0) out_row = base + (size_t)(((t / interval) - 1) % rows) * 14;
  out_row[0] = (double)t;
  out_row[1] = N;
  for (int a = 0; a < 3; ++a) {
    const double md = n ? acc[a] / N : 0.0, mx = n ? acc[6 + a] / N : 0.0;
    out_row[2 + a] = md;
    out_row[5 + a] = n ? acc[3 + a] / N - md * md : 0.0;
    out_row[8 + a] = mx;
    out_row[11 + a] = n ? acc[9 + a] / N - mx * mx : 0.0;
  }
  for (int m = 0; m < 12; ++m) acc[m] = 0.0;
}
__global__ void moments_finalize_kernel(double* acc, int64_t n, double* base, int interval, int rows,
                                        const int64_t* d_T, int toff) {
  moments_finalize_body(acc, n, base, interval, rows, d_T, toff);
}
__global__ void moments_batched(int finalize, const MomentArgs* __restrict__ args, const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const MomentArgs& a = args[m.domain];
  if (finalize) moments_finalize_body(a.acc, a.n, a.base, a.interval, a.rows, a.d_T, a.toff);
  else moments_body(a.pos, a.x0, a.n, a.acc, m.block, m.blocks);
}

int moments_grid(int64_t n) {
  const int64_t blocks = (n + 255) / 256;
  return (int)(blocks > 152 * 4 ? 152 * 4 : blocks);
}
void launch_moments(const float4* pos, const float4* x0, int64_t n, double* acc, double* base,
                    int interval, int rows, const int64_t* d_T, int toff, cudaStream_t st) {
  if (n > 0) moments_kernel<<<(unsigned)moments_grid(n), 256, 0, st>>>(pos, x0, n, acc);
  moments_finalize_kernel<<<1, 32, 0, st>>>(acc, n, base, interval, rows, d_T, toff);
}
size_t moments_args_size() { return sizeof(MomentArgs); }
void moments_args(void* dst, const float4* pos, const float4* x0, int64_t n, double* acc, double* base,
                  int interval, int rows, const int64_t* d_T, int toff) {
  *static_cast<MomentArgs*>(dst) = MomentArgs{pos, x0, n, acc, base, interval, rows, d_T, toff};
}
void launch_moments_batched(bool finalize, const void* args, const BlockMap* map, int nblocks, cudaStream_t st) {
  if (nblocks > 0)
    moments_batched<<<nblocks, 256, 0, st>>>(finalize ? 1 : 0, static_cast<const MomentArgs*>(args), map);
}

// ------------------------------------------------------------------------------------------
// Binning without allocation (rwmi_bin_walkers_noalloc). Its scratch -- per-walker ranks, per-cell
// offsets and the scan's block sums -- lives in this fixed device array instead of memory the
// caller or the library allocates; every GPU that loads the library holds it until exit.
// ------------------------------------------------------------------------------------------
constexpr int64_t NOALLOC_MAX_WALKERS = 1 << 20;
constexpr int64_t NOALLOC_MAX_CELLS = 1 << 20;
constexpr size_t NOALLOC_SCRATCH_WORDS =
    (size_t)NOALLOC_MAX_WALKERS + (size_t)NOALLOC_MAX_CELLS + (NOALLOC_MAX_CELLS + SCAN_TILE - 1) / SCAN_TILE + 1;
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

namespace {
std::mutex g_noalloc_mutex;
uint32_t* g_noalloc_addr[64] = {};   // device address of the scratch array, per device ordinal
thread_local char g_noalloc_err[256] = "";

rwmi_status noalloc_fail(rwmi_status s, const char* msg) {
  std::snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%s", msg);
  return s;
}
}  // namespace

const char* noalloc_last_error() { return g_noalloc_err; }

}  // namespace rwmi

extern "C" RWMI_API rwmi_status rwmi_bin_walkers_noalloc(const int32_t dims[3], uint32_t wall_mask,
                                                         const float* pos, int64_t n, float* pos_sorted,
                                                         uint32_t* counts, void* stream) {
  using namespace rwmi;
  if (!dims || !counts || (n > 0 && !pos) || wall_mask > 7)
    return noalloc_fail(RWMI_E_INVALID, "rwmi_bin_walkers_noalloc: null argument or bad wall mask");
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return noalloc_fail(RWMI_E_INVALID, "rwmi_bin_walkers_noalloc: dims must be >= 1");
    ncell *= dims[a];
  }
  if (ncell > NOALLOC_MAX_CELLS || n < 0 || n > NOALLOC_MAX_WALKERS)
    return noalloc_fail(RWMI_E_INVALID,
                        "rwmi_bin_walkers_noalloc: more than 1048576 cells or walkers (fixed scratch)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return noalloc_fail(RWMI_E_CUDA, "rwmi_bin_walkers_noalloc: no current CUDA device");
  uint32_t* scratch = nullptr;
  {
    // set-up, once per device with that device current: the host-side name of the array is a
    // stand-in, not a device address, so ask the runtime for the real one
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* addr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) {
        std::snprintf(g_noalloc_err, sizeof(g_noalloc_err), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return RWMI_E_CUDA;
      }
      g_noalloc_addr[dev] = (uint32_t*)addr;
    }
    scratch = g_noalloc_addr[dev];
  }
  uint32_t* rank = scratch;
  uint32_t* offsets = scratch + NOALLOC_MAX_WALKERS;
  uint32_t* bsums = offsets + NOALLOC_MAX_CELLS;
  Geom g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = dims[a];
    g.nb[a] = (dims[a] + BRICK - 1) / BRICK;
    g.wall[a] = (wall_mask >> a) & 1;
    g.inv_n[a] = 1.0f / (float)dims[a];
  }
  g.nxy = (uint32_t)dims[0] * (uint32_t)dims[1];
  g.ncell = (uint32_t)ncell;
  g.ncell_pad = (uint32_t)ncell;
  make_divisor((uint32_t)dims[0], g.mx, g.sx);
  make_divisor(g.nxy, g.mxy, g.sxy);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)ncell, st);
  if (e == cudaSuccess && n > 0) {
    const float4* p4 = reinterpret_cast<const float4*>(pos);
    launch_histogram(g, p4, n, counts, pos_sorted ? rank : nullptr, st);
    if (pos_sorted) {
      launch_scan(counts, offsets, bsums, (uint32_t)ncell, st);
      launch_scatter_pos(g, p4, n, offsets, rank, reinterpret_cast<float4*>(pos_sorted), st);
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    std::snprintf(g_noalloc_err, sizeof(g_noalloc_err), "rwmi_bin_walkers_noalloc: %s", cudaGetErrorString(e));
    return RWMI_E_CUDA;
  }
  return RWMI_OK;
}
