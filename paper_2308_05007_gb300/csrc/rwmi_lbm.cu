// rwmi_lbm.cu -- the fused LBM step: pull stream (periodic wrap / half-way bounce-back) + BGK
// collide (Eqs. 12-15) with Guo forcing and either PSM solid coupling or the paper's
// interpolated bounce-back (Eqs. 23-27); writes the populations, the velocity field and, on
// reduction steps, per-particle force/torque and the FP64 sums.
//   lbm_kernel        the update (one cell per thread, direct coalesced pulls), the fused update +
//                     reduction of reduction steps (binary32-shifted and binary64 storage, every
//                     free-DEM step) and a reduce-only pass (the other storages, staged updates)
//   lbm_batched       the same update over the cells of many domains (fused batch)
//   lbm_tma_kernel    the update with its pulled rows staged by TMA tensor copies (an option)
//   ibb_links_kernel  IBB node words and link list; ibb_link_kernel: q and G of every link
#include <atomic>
#include <type_traits>

#include "rwmi_lattice.cuh"

namespace rwmi {

// ------------------------------------------------------------------------------------------
// Fused pull-stream + collide (Eqs. 12-15), partially saturated cells, Guo forcing.
// One thread per cell, flat index c = x + nx (y + ny z); direction planes are contiguous, so
// every pull load of a warp is one (shifted) coalesced row segment. Storage: binary32 f_i,
// binary32 f_i - w_i rho0 ("shifted") or binary16 shifted, with binary32 arithmetic; or
// binary64 shifted with binary64 arithmetic.
// ------------------------------------------------------------------------------------------
// Base pointers of the Q direction planes (kernel parameters: constant-bank operands, so each
// access is one address multiply-add).
template <int Q, typename T> struct Planes {
  const T* in[Q];
  T* out[Q];
};

// q of Eq. 25: 24 binary32 bisection steps on Eq. 3 of one particle along x_f + s e, s in [0, 1]
// (the CPU oracle's sequence: midpoint 0.5 (lo + hi), point x_f + mid e), q = the bracket's
// middle. ibb_link_kernel calls it once per link (listed, or in an overflow slot).
__device__ __forceinline__ float ibb_link_q(const float4* __restrict__ cw, int c0, int c1, float x0, float y0,
                                         float z0, int ex, int ey, int ez, const Geom& g) {
  float lo = 0.0f, hi = 1.0f;
  for (int it = 0; it < 24; ++it) {
    const float mid = __fmul_rn(0.5f, __fadd_rn(lo, hi));
    const float xm = __fadd_rn(x0, __fmul_rn(mid, (float)ex));
    const float ym = __fadd_rn(y0, __fmul_rn(mid, (float)ey));
    const float zm = __fadd_rn(z0, __fmul_rn(mid, (float)ez));
    if (metaball_exact(cw, c0, c1, xm, ym, zm, g) >= 1.0f) hi = mid; else lo = mid;
  }
  return __fmul_rn(0.5f, __fadd_rn(lo, hi));
}

// Guo pair constant j (0: 9 w_i g e_i.F, 1: 3 w_i g e_i.F) of the opposite pair (i, i + H) at the
// update's time, in the arithmetic type (both of a pair come from one 8- or 16-byte load)
template <typename R>
__device__ __forceinline__ R gk_pair(const StepParams* __restrict__ sp, int i, int j) {
  if constexpr (sizeof(R) == 8) {
    const double2 v = reinterpret_cast<const double2*>(guo_pairs(sp)->kd)[i - 1];
    return j ? v.y : v.x;
  } else {
    const float2 v = reinterpret_cast<const float2*>(guo_pairs(sp)->k)[i - 1];
    return j ? v.y : v.x;
  }
}

// Row tiles of the TMA-staged update (lbm_tma_kernel): TMA_BX cells of one x-row per tile. Each
// direction's source row is copied with a halo of 16 bytes on both sides, so that the copy
// starts on a 16-byte boundary (x0 - halo) and covers x0 - 1 .. x0 + TMA_BX; rows sit 128-byte
// aligned in shared memory.
constexpr int TMA_BX = 128;
template <int STORE> struct TmaRow {
  static constexpr int es = (int)sizeof(typename Store<STORE>::T);
  static constexpr int halo = 16 / es;                                  // elements
  static constexpr int box = TMA_BX + 2 * halo;                         // elements copied per row
  static constexpr int bytes = box * es;                                // a multiple of 16
  static constexpr int pad = ((bytes + 127) / 128) * 128 / es;          // elements between rows
};

// Flat offset of the pull source x - e_d of cell (x, y, z) for a run-time direction d (periodic
// wrap); false where x - e_d lies beyond a plane wall.
template <int Q, bool WALLS>
__device__ __forceinline__ bool pull_source(const Geom& g, uint32_t x, uint32_t y, uint32_t z, int d, int& off) {
  using L = Lat<Q>;
  const int ex = L::e(d, 0), ey = L::e(d, 1), ez = L::e(d, 2);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int sy = nx, sz = (int)g.nxy;
  if (WALLS && ((g.wall[0] && ((ex > 0 && x == 0) || (ex < 0 && (int)x == nx - 1))) ||
                (g.wall[1] && ((ey > 0 && y == 0) || (ey < 0 && (int)y == ny - 1))) ||
                (g.wall[2] && ((ez > 0 && z == 0) || (ez < 0 && (int)z == nz - 1)))))
    return false;
  off = (ex > 0 ? (x == 0 ? nx - 1 : -1) : ex < 0 ? ((int)x == nx - 1 ? -(nx - 1) : 1) : 0) +
        (ey > 0 ? (y == 0 ? (ny - 1) * sy : -sy) : ey < 0 ? ((int)y == ny - 1 ? -(ny - 1) * sy : sy) : 0) +
        (ez > 0 ? (z == 0 ? (nz - 1) * sz : -sz) : ez < 0 ? ((int)z == nz - 1 ? -(nz - 1) * sz : sz) : 0);
  return true;
}

// One IBB link (Eqs. 23-25): fluid node x_f = cell c at (x, y, z), direction i whose source
// x_f - e_i is a solid node of particle p, wall distance qf. rho_f and u_f are x_f's own
// post-collision density and previous velocity. Returns G_i(x_f) = G^eq_ip(rho_f, u_d) +
// G^neq_ip(x_f) + 6 w rho_f e_i.u_w (the storage shift cancels); Gp = G+_ip(x_f), the wall point
// xw and its rigid velocity uw are left for the momentum exchange.
template <int Q, int STORE, bool WALLS>
__device__ __forceinline__ typename Store<STORE>::R
ibb_link_value(const Geom& g, const typename Store<STORE>::T* __restrict__ in0, const float4* __restrict__ uprev,
               const uint16_t* __restrict__ nodes, const PoseF* __restrict__ pose, const PoseD* __restrict__ posed,
               int c, uint32_t x, uint32_t y, uint32_t z, int i, int p, typename Store<STORE>::R qf,
               typename Store<STORE>::R rho_f, const typename Store<STORE>::R (&uf)[3],
               typename Store<STORE>::R& Gp, typename Store<STORE>::R (&xw)[3], typename Store<STORE>::R (&uw)[3]) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  const int ip = L::opp(i);
  const int ex = L::e(ip, 0), ey = L::e(ip, 1), ez = L::e(ip, 2);   // into the wall
  xw[0] = (R)x + R(0.5) + qf * (R)ex;
  xw[1] = (R)y + R(0.5) + qf * (R)ey;
  xw[2] = (R)z + R(0.5) + qf * (R)ez;
  rigid_velocity<R>(g, pose, posed, p, xw[0], xw[1], xw[2], uw);
  R uff[3] = {uf[0], uf[1], uf[2]};
  int off = 0;
  if (pull_source<Q, WALLS>(g, x, y, z, ip, off)) {   // x_ff = x_f + e_i, unless solid or beyond a wall
    const int cf = c + off;
    if (nodes[cf] == 0) {
      const float4 v = uprev[cf];
      uff[0] = (R)v.x; uff[1] = (R)v.y; uff[2] = (R)v.z;
    }
  }
  R ud[3];
  for (int a = 0; a < 3; ++a) {
    const R us1 = qf <= R(0.5) ? R(2) * qf * uf[a] + (R(1) - R(2) * qf) * uff[a]
                               : (R(1) - qf) / qf * uf[a] + (R(2) * qf - R(1)) / qf * uw[a];
    const R us2 = (R(1) - qf) / (R(1) + qf) * uff[a] + R(2) * qf / (R(1) + qf) * uw[a];
    ud[a] = us1 / R(3) + R(2) * us2 / R(3);
  }
  const R w = L::template wt<R>(ip);
  const R eud = (R)ex * ud[0] + (R)ey * ud[1] + (R)ez * ud[2];
  const R euf = (R)ex * uf[0] + (R)ey * uf[1] + (R)ez * uf[2];
  const R uud = ud[0] * ud[0] + ud[1] * ud[1] + ud[2] * ud[2];
  const R uuf = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
  const R euw = -((R)ex * uw[0] + (R)ey * uw[1] + (R)ez * uw[2]);   // e_i . u_w, e_i = -e_ip
  Gp = S::ld(in0 + (size_t)ip * g.ncell_pad + c);
  return Gp + w * rho_f * (R(3) * (eud - euf) + R(4.5) * (eud * eud - euf * euf) - R(1.5) * (uud - uuf)) +
         R(6) * w * rho_f * euw;
}

// Momentum exchange of one link on its particle p (Galilean invariant, Section 2.4.3):
// (e_ip - u_w) G+_ip - (e_i - u_w) G_i, and its torque about p's origin (minimum image).
template <int Q, int STORE>
__device__ __forceinline__ void ibb_link_force(const Geom& g, const PoseF* __restrict__ pose,
                                               const PoseD* __restrict__ posed, int i, int p,
                                               typename Store<STORE>::R rho0, typename Store<STORE>::R Gp,
                                               typename Store<STORE>::R G, const typename Store<STORE>::R (&xw)[3],
                                               const typename Store<STORE>::R (&uw)[3],
                                               typename Store<STORE>::R (&Fl)[3], typename Store<STORE>::R (&Tl)[3]) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  const int ip = L::opp(i);
  const R ex = (R)L::e(ip, 0), ey = (R)L::e(ip, 1), ez = (R)L::e(ip, 2);
  const R w = L::template wt<R>(ip);
  const R sh = S::shifted ? w * rho0 : R(0);
  const R gp = Gp + sh, gi = G + sh;
  Fl[0] = (ex - uw[0]) * gp - (-ex - uw[0]) * gi;
  Fl[1] = (ey - uw[1]) * gp - (-ey - uw[1]) * gi;
  Fl[2] = (ez - uw[2]) * gp - (-ez - uw[2]) * gi;
  R po[3], pv[3], pw[3];
  load_pose<R>(pose, posed, p, po, pv, pw);
  R r[3] = {xw[0] - po[0], xw[1] - po[1], xw[2] - po[2]};
  for (int a = 0; a < 3; ++a)
    if (!g.wall[a]) {
      const R na = (R)g.n[a];
      if (r[a] > R(0.5) * na) r[a] -= na; else if (r[a] < -R(0.5) * na) r[a] += na;
    }
  Tl[0] = r[1] * Fl[2] - r[2] * Fl[1];
  Tl[1] = r[2] * Fl[0] - r[0] * Fl[2];
  Tl[2] = r[0] * Fl[1] - r[1] * Fl[0];
}

// Momentum exchange of one cell's links, in direction order (Section 2.4.3): q and G of each link
// from the link list (k0 >= 0: the cell's links at k0, k0 + 1, ...) or from the overflow table
// (k0 < 0: slot -1 - k0, link i at cap + slot (Q - 1) + i - 1); per-particle sums in Fib/Tib for
// the cell's first particle, direct atomics for a second particle at one node (rare).
template <int Q, int STORE>
__device__ __forceinline__ void ibb_cell_force(const Geom& g, const typename Store<STORE>::T* __restrict__ in0,
                                               const PoseF* __restrict__ pose, const PoseD* __restrict__ posed,
                                               const uint16_t* __restrict__ nodes, int c, uint32_t x, uint32_t y,
                                               uint32_t z, unsigned lmask, int k0, int cap,
                                               const float* __restrict__ ib_q,
                                               const typename Store<STORE>::R* __restrict__ ib_g,
                                               typename Store<STORE>::R rho0,
                                               double* __restrict__ forces, int& owner,
                                               typename Store<STORE>::R (&Fib)[3], typename Store<STORE>::R (&Tib)[3]) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  const bool ovf = k0 < 0;
  const int kb = ovf ? cap + (-1 - k0) * (Q - 1) : k0;
  int k = kb;
  for (unsigned m = lmask; m; m &= m - 1u, ++k) {
    const int i = __ffs(m) - 1, ip = L::opp(i);
    const int kk = ovf ? kb + i - 1 : k;
    int off = 0;
    pull_source<Q, true>(g, x, y, z, i, off);   // a link's source is never beyond a wall
    const int p = (int)nodes[c + off] - 1;
    const R qf = (R)ib_q[kk];
    const R G = ib_g[kk];
    const int ex = L::e(ip, 0), ey = L::e(ip, 1), ez = L::e(ip, 2);
    const R xw[3] = {(R)x + R(0.5) + qf * (R)ex, (R)y + R(0.5) + qf * (R)ey, (R)z + R(0.5) + qf * (R)ez};
    R uw[3];
    rigid_velocity<R>(g, pose, posed, p, xw[0], xw[1], xw[2], uw);
    const R Gp = S::ld(in0 + (size_t)ip * g.ncell_pad + c);
    R Fl[3], Tl[3];
    ibb_link_force<Q, STORE>(g, pose, posed, i, p, rho0, Gp, G, xw, uw, Fl, Tl);
    if (owner < 0 || owner == p) {
      owner = p;
      for (int a = 0; a < 3; ++a) { Fib[a] += Fl[a]; Tib[a] += Tl[a]; }
    } else {
      for (int a = 0; a < 3; ++a) {
        atomicAdd(&forces[6 * p + a], (double)Fl[a]);
        atomicAdd(&forces[6 * p + 3 + a], (double)Tl[a]);
      }
    }
  }
}

// IBB: the paper's coupling (Section 2.4.3) instead of partially saturated cells. A cell of a
// flagged brick reads its node class; a solid node holds the equilibrium at its particle's rigid
// velocity; a fluid node replaces the population pulled from each solid neighbour by Eqs. 23-25
// (q by the same binary32 bisection as the CPU oracle) and, on reduction steps, adds the
// Galilean-invariant momentum exchange of the link to its particle's force and torque.
// MODE 0: the update. MODE 2: update and reduction in one pass, on the steps whose sums are read
// (binary32-shifted and binary64 storage) and on every free-DEM step. Its update arithmetic
// stores the same bits as MODE 0 (a GPU test checks every instantiation that uses it), so
// reducing and non-reducing steps agree bit for bit. MODE 1: a reduce-only pass for the other
// storages and the staged update; it runs after the update, re-pulls the same input populations,
// forms the FP64 sums and particle forces, and stores nothing.
template <int Q, int STORE, bool WALLS, int MODE, bool IBB, bool STAGED = false>
__device__ __forceinline__ void lbm_body(Geom g, Planes<Q, typename Store<STORE>::T> pl,
                                                  float4* __restrict__ u4,
                                                  const uint16_t* __restrict__ solid,
                                                  const uint32_t* __restrict__ bword,
                                                  const PoseF* __restrict__ pose,
                                                  const PoseD* __restrict__ posed,
                                                  const StepParams* __restrict__ sp,
                                                  typename Store<STORE>::R tau,
                                                  typename Store<STORE>::R omega,
                                                  typename Store<STORE>::R guo0,
                                                  typename Store<STORE>::R rho0, double* __restrict__ red,
                                                  double* __restrict__ forces,
                                                  const uint16_t* __restrict__ nodes,
                                                  const float4* __restrict__ uprev,
                                                  const ParticleDesc* __restrict__ desc,
                                                  const float4* __restrict__ cworld,
                                                  const int32_t* __restrict__ ib_base,
                                                  const uint32_t* __restrict__ ib_word,
                                                  const float* __restrict__ ib_q,
                                                  const typename Store<STORE>::R* __restrict__ ib_g, int ib_cap,
                                                  int blk, const typename Store<STORE>::T* srow = nullptr,
                                                  uint32_t staged_idx = 0, bool staged_valid = false,
                                                  int staged_lx = 0) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;   // arithmetic type: binary32, or binary64 for the binary64 storage
  constexpr bool REDUCE = MODE != 0, STORES = MODE != 1;
  // Guo pair constants loaded (one multiply-add per pair) or formed from F in each thread: the
  // loaded form measured faster for D3Q19 and binary32-shifted D3Q15, slower for binary16 and
  // plain binary32 D3Q15 (more spilled registers at 40)
  constexpr bool GK_CONST = !(Q == 15 && (STORE == 0 || STORE == 2));
  // tau, omega = 1/tau, guo0 = 1 - 1/(2 tau) and rho0 arrive in R (formed and converted on the
  // host: per-thread divisions and binary64 -> binary32 conversions cost issue slots, and the
  // conversions occupy GB300's narrow FP64 pipe)
  // STAGED (lbm_tma_kernel): the cell and its valid flag come from the row tile, and pulls read
  // the tile's rows in shared memory (srow: direction i at i * TmaRow<STORE>::pad elements, the
  // cell's own source at TmaRow<STORE>::halo + staged_lx - e_x)
  const uint32_t idx = STAGED ? staged_idx : blk * blockDim.x + threadIdx.x;
  const bool valid = STAGED ? staged_valid : idx < g.ncell;
  const int c = (int)(valid || STAGED ? idx : g.ncell - 1);   // tail lanes recompute the last cell and store
  const int cs = valid ? c : (int)g.ncell_pad - 1;  // into the spare slot no cell owns (no branches)
  const uint32_t z = fast_div((uint32_t)c, g.mxy, g.sxy);
  const uint32_t rem = (uint32_t)c - z * g.nxy;
  const uint32_t y = fast_div(rem, g.mx, g.sx);
  const uint32_t x = rem - y * g.n[0];
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int sy = nx, sz = (int)g.nxy;
  // source offsets for e_a = +1 (source at -1) and e_a = -1 (source at +1), periodic wrap
  const int ox_p = x == 0 ? nx - 1 : -1, ox_m = (int)x == nx - 1 ? -(nx - 1) : 1;
  const int oy_p = y == 0 ? (ny - 1) * sy : -sy, oy_m = (int)y == ny - 1 ? -(ny - 1) * sy : sy;
  const int oz_p = z == 0 ? (nz - 1) * sz : -sz, oz_m = (int)z == nz - 1 ? -(nz - 1) * sz : sz;
  R f[Q];
  bool wall_cell = false;
  if (WALLS)
    wall_cell = (g.wall[0] && (x == 0 || (int)x == nx - 1)) || (g.wall[1] && (y == 0 || (int)y == ny - 1)) ||
                (g.wall[2] && (z == 0 || (int)z == nz - 1));
  if (!wall_cell) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
      if constexpr (STAGED) {
        f[i] = S::ld(srow + i * TmaRow<STORE>::pad + (TmaRow<STORE>::halo + staged_lx - ex));
      } else {
        const int off = (ex > 0 ? ox_p : ex < 0 ? ox_m : 0) + (ey > 0 ? oy_p : ey < 0 ? oy_m : 0) +
                        (ez > 0 ? oz_p : ez < 0 ? oz_m : 0);
        f[i] = S::ld(pl.in[i] + (c + off));
      }
    }
  } else {   // half-way bounce-back where x - e_i lies beyond a wall: f_i(x) = f+_opp(i)(x)
    const bool bx_p = g.wall[0] && x == 0, bx_m = g.wall[0] && (int)x == nx - 1;
    const bool by_p = g.wall[1] && y == 0, by_m = g.wall[1] && (int)y == ny - 1;
    const bool bz_p = g.wall[2] && z == 0, bz_m = g.wall[2] && (int)z == nz - 1;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
      const int off = (ex > 0 ? ox_p : ex < 0 ? ox_m : 0) + (ey > 0 ? oy_p : ey < 0 ? oy_m : 0) +
                      (ez > 0 ? oz_p : ez < 0 ? oz_m : 0);
      const bool wb = (ex > 0 && bx_p) || (ex < 0 && bx_m) || (ey > 0 && by_p) || (ey < 0 && by_m) ||
                      (ez > 0 && bz_p) || (ez < 0 && bz_m);
      if constexpr (STAGED)
        f[i] = wb ? S::ld(pl.in[L::opp(i)] + c)
                  : S::ld(srow + i * TmaRow<STORE>::pad + (TmaRow<STORE>::halo + staged_lx - ex));
      else
        f[i] = wb ? S::ld(pl.in[L::opp(i)] + c) : S::ld(pl.in[i] + (c + off));
    }
  }
  // ---- the paper's coupling: IBB links of a fluid node next to solid nodes (Eqs. 23-25) ----
  bool solid_self = false;
  R Fib[3] = {R(0), R(0), R(0)}, Tib[3] = {R(0), R(0), R(0)};   // IBB: this cell's link forces
  int ib_owner = -1;
  if constexpr (IBB) {
    // ibb_links_kernel, which ran before, left every cell of a flagged brick its node word: bit 0
    // a solid node, bit i a link (x - e_i a solid node, not beyond a wall), and ibb_link_kernel
    // left q and G_i of every link. Cells of other bricks have no solid neighbour (the IBB brick
    // radius is at least rb + sqrt 3).
    unsigned lmask = 0u;
    const uint32_t bq = ((z >> 3) * (uint32_t)g.nb[1] + (y >> 3)) * (uint32_t)g.nb[0] + (x >> 3);
    if (valid && (bword[bq] >> 16)) {
      const uint32_t lw = ib_word[c];
      solid_self = (lw & 1u) != 0u;
      lmask = lw & ~1u;
    }
    // the cell's links: in the list at ib_base[c] in direction order, or, for a cell whose links
    // did not fit in the list, in its overflow slot -1 - ib_base[c] by direction
    if (lmask) {
      const int k0 = ib_base[c];
      const bool ovf = k0 < 0;
      const int kb = ovf ? ib_cap + (-1 - k0) * (Q - 1) : k0;
      int k = kb;
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if ((lmask >> i) & 1u) {
          f[i] = ib_g[ovf ? kb + i - 1 : k];
          ++k;
        }
      if (REDUCE) ibb_cell_force<Q, STORE>(g, pl.in[0], pose, posed, nodes, c, x, y, z, lmask, k0, ib_cap, ib_q, ib_g,
                                           rho0, forces, ib_owner, Fib, Tib);
    }
  }
  // moments (Eqs. 14-15); with shifted storage f holds f_i - w_i rho0
  R drho = R(0.0), jx = R(0.0), jy = R(0.0), jz = R(0.0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    drho += f[i];
    if (L::e(i, 0)) jx += L::e(i, 0) * f[i];
    if (L::e(i, 1)) jy += L::e(i, 1) * f[i];
    if (L::e(i, 2)) jz += L::e(i, 2) * f[i];
  }
  const R rho = S::shifted ? rho0 + drho : drho;
  R Fx, Fy, Fz;
  if constexpr (GK_CONST && sizeof(R) == 4) {   // F and its pad as one 16-byte load (byte 0 of
    const float4 F4 = *reinterpret_cast<const float4*>(sp->F);   // a cudaMalloc'd StepParams)
    Fx = F4.x; Fy = F4.y; Fz = F4.z;
  } else {
    Fx = sizeof(R) == 8 ? (R)sp->Fd[0] : (R)sp->F[0];
    Fy = sizeof(R) == 8 ? (R)sp->Fd[1] : (R)sp->F[1];
    Fz = sizeof(R) == 8 ? (R)sp->Fd[2] : (R)sp->F[2];
  }
  // 1/rho correctly rounded (as the IEEE division 1/rho): a biased reciprocal would act like a
  // small momentum sink every step, which a steady forced flow amplifies by ~1/(tau nu k^2)
  const R inv_rho = sizeof(R) == 8 ? R(1.0) / rho : (R)__frcp_rn((float)rho);
  const R ux = (jx + R(0.5) * Fx) * inv_rho, uy = (jy + R(0.5) * Fy) * inv_rho,
              uz = (jz + R(0.5) * Fz) * inv_rho;
  const R uu = ux * ux + uy * uy + uz * uz;
  // partially saturated cell: solid word valid only in bricks flagged for this time. Under IBB
  // (B = 0) us is a solid node's rigid velocity.
  R B = R(0.0), usx = R(0.0), usy = R(0.0), usz = R(0.0);
  int owner = -1;
  if constexpr (IBB) {
    if (solid_self) {
      R us[3];
      rigid_velocity<R>(g, pose, posed, (int)nodes[c] - 1, (R)x + R(0.5), (R)y + R(0.5), (R)z + R(0.5), us);
      usx = us[0]; usy = us[1]; usz = us[2];
    }
  } else {
    const uint32_t b = ((z >> 3) * (uint32_t)g.nb[1] + (y >> 3)) * (uint32_t)g.nb[0] + (x >> 3);
    if (bword[b] >> 16) {
      const uint16_t sw = solid[c];
      const int cnt = sw & 0x7f;
      if (cnt && valid) {
        owner = sw >> 7;
        const R eps = (R)cnt * (R(1.0) / R(64.0));
        B = eps * (tau - R(0.5)) / ((R(1.0) - eps) + (tau - R(0.5)));
        R po[3], pv[3], pw[3];
        load_pose<R>(pose, posed, owner, po, pv, pw);
        R r[3] = {(R)x + R(0.5) - po[0], (R)y + R(0.5) - po[1], (R)z + R(0.5) - po[2]};
        for (int a = 0; a < 3; ++a)
          if (!g.wall[a]) {
            const R na = (R)g.n[a];
            if (r[a] > R(0.5) * na) r[a] -= na; else if (r[a] < -R(0.5) * na) r[a] += na;
          }
        usx = pv[0] + pw[1] * r[2] - pw[2] * r[1];
        usy = pv[1] + pw[2] * r[0] - pw[0] * r[2];
        usz = pv[2] + pw[0] * r[1] - pw[1] * r[0];
      }
    }
  }
  // BGK with Guo forcing (Eqs. 12-13), per direction i:
  //   f+_i = (1 - rtau) f_i + rtau feq_i + guo w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)],
  // rtau = (1 - B) / tau, guo = (1 - B)(1 - 1/(2 tau)), with 1/tau and 1 - 1/(2 tau) from the host,
  // feq_i = w_i rho' + w_i rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u), rho' = rho - rho0 when shifted.
  // An opposite pair (i, i') shares e.u, (e.u)^2 and the even parts. The equilibrium keeps
  // w_i rho' apart from w_i rho times the velocity polynomial: grouped otherwise (e.g. folding
  // rho' into the velocity terms) the binary32 rounding of a steady forced flow grew the
  // velocity error against the FP64 oracle from 0.96e-5 to 1.5e-5 over 500 steps.
  // a solid node (IBB) holds the equilibrium at its particle's rigid velocity and rho0
  auto solid_eq = [&](R w, R eu, R uus) {
    const R dev = R(3) * eu + R(4.5) * eu * eu - R(1.5) * uus;
    return S::shifted ? w * rho0 * dev : w * rho0 * (R(1) + dev);
  };
  const R omB = R(1.0) - B;
  const R rtau = omB * omega;
  const R guo = omB * guo0;
  const R om1 = R(1.0) - rtau;
  const R uF = ux * Fx + uy * Fy + uz * Fz;
  const R usus = usx * usx + usy * usy + usz * usz;
  const R m15uu = -R(1.5) * uu;
  R dpx = R(0.0), dpy = R(0.0), dpz = R(0.0);
  R out[Q];
  {  // rest direction; its own opposite: Omega_0 = feq_0(rho, u_s) - feq_0(rho, u)
    const R w = L::template wt<R>(0);
    const R feq0 = w * (S::shifted ? drho : rho) + (w * rho) * m15uu;
    out[0] = om1 * f[0] + (rtau * feq0 + (w * guo) * (-R(3.0) * uF)) + B * (R(1.5) * w * rho * (uu - usus));
    if (IBB && solid_self) out[0] = solid_eq(w, R(0), usus);
  }
  // opposite pairs (i, i + H) share e.u. One warp-uniform branch picks the loop with the solid
  // terms of partially saturated cells (lanes with B = 0 add exact zeros there) or the plain one;
  // under IBB another picks the loop that gives solid nodes their rigid equilibrium.
  auto pair_update = [&](auto psm, auto sol) {
#pragma unroll
    for (int i = 1; i <= L::H; ++i) {
      const int io = i + L::H;
      const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
      const R w = L::template wt<R>(i);
      const R eu = ex * ux + ey * uy + ez * uz;
      // Guo term: even part 9 w g (e.u)(e.F) - 3 w g u.F, odd part 3 w g e.F (g = 1 - 1/(2 tau)),
      // times 1 - B in partially saturated cells
      if constexpr (GK_CONST) {   // from the pair constants of this time
        const R wdr = w * (S::shifted ? drho : rho), wr = w * rho;
        const R sym = R(4.5) * eu * eu + m15uu;        // even part of the velocity polynomial
        const R feq_p = wdr + wr * (sym + R(3.0) * eu);
        const R feq_m = wdr + wr * (sym - R(3.0) * eu);
        const R k9 = gk_pair<R>(sp, i, 0), k3 = gk_pair<R>(sp, i, 1);
        const R Se = k9 * eu + (R(-3.0) * (w * guo0)) * uF;
        R gp = Se + k3, gm = Se - k3;
        if constexpr (decltype(psm)::value) {
          gp *= omB;
          gm *= omB;
        }
        out[i] = om1 * f[i] + (rtau * feq_p + gp);
        out[io] = om1 * f[io] + (rtau * feq_m + gm);
      } else {                    // from F in every thread (the same statements, in this order)
        const R eF = ex * Fx + ey * Fy + ez * Fz;
        const R wdr = w * (S::shifted ? drho : rho), wr = w * rho, wg = w * guo;
        const R sym = R(4.5) * eu * eu + m15uu;
        const R feq_p = wdr + wr * (sym + R(3.0) * eu);
        const R feq_m = wdr + wr * (sym - R(3.0) * eu);
        const R Se = wg * (R(9.0) * (eu * eF) - R(3.0) * uF);
        const R So = (R(3.0) * wg) * eF;
        out[i] = om1 * f[i] + (rtau * feq_p + (Se + So));
        out[io] = om1 * f[io] + (rtau * feq_m + (Se - So));
      }
      const R wr = w * rho;
      if constexpr (decltype(psm)::value) {
        const R eus = ex * usx + ey * usy + ez * usz;
        const R common = wr * (R(4.5) * (eus * eus - eu * eu) - R(1.5) * (usus - uu));
        const R odd = wr * R(3.0) * (eu + eus);
        const R om_p = (f[io] - f[i]) + odd + common;   // Omega_i
        const R om_m = (f[i] - f[io]) - odd + common;   // Omega_opp(i)
        out[i] += B * om_p;
        out[io] += B * om_m;
        const R dm = B * (om_p - om_m);                 // B (Omega_i e_i + Omega_opp e_opp) / e_i
        dpx += dm * ex; dpy += dm * ey; dpz += dm * ez;
      }
      if constexpr (decltype(sol)::value) {
        if (solid_self) {
          const R eus = (R)ex * usx + (R)ey * usy + (R)ez * usz;
          out[i] = solid_eq(w, eus, usus);
          out[io] = solid_eq(w, -eus, usus);
        }
      }
      if (STORES) {   // stored at once: fewer values live at the same time
        S::st(pl.out[i] + cs, out[i]);
        S::st(pl.out[io] + cs, out[io]);
      }
    }
  };
  if (IBB) {
    if (__any_sync(0xffffffffu, solid_self)) pair_update(std::false_type{}, std::true_type{});
    else pair_update(std::false_type{}, std::false_type{});
  } else if (!__any_sync(0xffffffffu, B > R(0.0))) {
    pair_update(std::false_type{}, std::false_type{});
  } else {
    pair_update(std::true_type{}, std::false_type{});
  }
  if (STORES) {   // the reduce-only pass stores nothing
    S::st(pl.out[0] + cs, out[0]);
    if (IBB && solid_self) u4[cs] = make_float4((float)usx, (float)usy, (float)usz, (float)rho0);
    else u4[cs] = make_float4((float)ux, (float)uy, (float)uz, (float)rho);
  }
  // hydrodynamic force on the owner particle: -B sum_i Omega_i e_i; torque about its origin.
  // Formed, like the mass/momentum sums, only on the step whose sums are read (REDUCE); the
  // accumulators of every other step are cleared again before anyone reads them.
  const unsigned full = 0xffffffffu;
  const bool hasF = IBB ? (ib_owner >= 0) : (owner >= 0);
  if (IBB) owner = ib_owner;
  if (REDUCE && __any_sync(full, hasF)) {
    R Fc[3] = {-dpx, -dpy, -dpz};
    R Tc[3] = {R(0.0), R(0.0), R(0.0)};
    if (IBB) {   // link forces and torques of the cell
      for (int a = 0; a < 3; ++a) { Fc[a] = Fib[a]; Tc[a] = Tib[a]; }
    } else if (hasF) {
      R po[3], pv[3], pw[3];
      load_pose<R>(pose, posed, owner, po, pv, pw);
      R r[3] = {(R)x + R(0.5) - po[0], (R)y + R(0.5) - po[1], (R)z + R(0.5) - po[2]};
      for (int a = 0; a < 3; ++a)
        if (!g.wall[a]) {
          const R na = (R)g.n[a];
          if (r[a] > R(0.5) * na) r[a] -= na; else if (r[a] < -R(0.5) * na) r[a] += na;
        }
      Tc[0] = r[1] * Fc[2] - r[2] * Fc[1];
      Tc[1] = r[2] * Fc[0] - r[0] * Fc[2];
      Tc[2] = r[0] * Fc[1] - r[1] * Fc[0];
    }
    const int key = hasF ? owner : -1;
    const int first = __shfl_sync(full, key, __ffs(__ballot_sync(full, hasF)) - 1);
    const bool uniform = __all_sync(full, !hasF || key == first);
    if (uniform) {
      R v[6] = {Fc[0], Fc[1], Fc[2], Tc[0], Tc[1], Tc[2]};
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        if (!hasF) v[m] = R(0.0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(full, v[m], o);
      }
      if ((threadIdx.x & 31) == 0)
        for (int m = 0; m < 6; ++m) atomicAdd(&forces[6 * first + m], (double)v[m]);
    } else if (hasF) {
      for (int m = 0; m < 3; ++m) {
        atomicAdd(&forces[6 * owner + m], (double)Fc[m]);
        atomicAdd(&forces[6 * owner + 3 + m], (double)Tc[m]);
      }
    }
  }
  if (REDUCE) {   // sums of (rho - rho0) and sum_i f_i e_i (pre-collision): the arithmetic type
                  // within the block (256 small deviations), FP64 across blocks (GB300's FP64
                  // pipe is narrow)
    const bool fl = valid && !solid_self;   // fluid nodes only (solid nodes: IBB)
    R v[4] = {fl ? (S::shifted ? drho : rho - rho0) : R(0.0), fl ? jx : R(0.0),
                  fl ? jy : R(0.0), fl ? jz : R(0.0)};
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(full, v[m], o);
    __shared__ R s_red[8][4];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
      for (int m = 0; m < 4; ++m) s_red[wid][m] = v[m];
    __syncthreads();
    if (threadIdx.x < 4) {   // striped slots keep the FP64 atomics of 65536 blocks uncontended
      R s = R(0.0);
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w][threadIdx.x];
      atomicAdd(&red[4 * (blk % RED_SLOTS) + threadIdx.x], (double)s);
    }
  }
}

// Arguments of one LBM launch (the partially saturated cells; the IBB inputs stay null).
template <int Q, int STORE> struct LbmArgs {
  using T = typename Store<STORE>::T;
  using R = typename Store<STORE>::R;
  Geom g;
  Planes<Q, T> pl;
  float4* u4;
  const uint16_t* solid;
  const uint32_t* bword;
  const PoseF* pose;
  const PoseD* posed;
  const StepParams* sp;
  R tau, omega, guo0, rho0;
  double* red;
  double* forces;
};

#define RWMI_LBM_BOUNDS __launch_bounds__(256, sizeof(typename Store<STORE>::R) == 8 ? 2 : IBB ? (MODE == 0 ? 6 : 4) : (Q == 19 ? 5 : 6))

template <int Q, int STORE, bool WALLS, int MODE, bool IBB>
__global__ void RWMI_LBM_BOUNDS
lbm_kernel(Geom g, Planes<Q, typename Store<STORE>::T> pl, float4* __restrict__ u4, const uint16_t* __restrict__ solid,
           const uint32_t* __restrict__ bword, const PoseF* __restrict__ pose, const PoseD* __restrict__ posed,
           const StepParams* __restrict__ sp, typename Store<STORE>::R tau, typename Store<STORE>::R omega,
           typename Store<STORE>::R guo0, typename Store<STORE>::R rho0, double* __restrict__ red,
           double* __restrict__ forces, const uint16_t* __restrict__ nodes, const float4* __restrict__ uprev,
           const ParticleDesc* __restrict__ desc, const float4* __restrict__ cworld,
           const int32_t* __restrict__ ib_base, const uint32_t* __restrict__ ib_word, const float* __restrict__ ib_q,
           const typename Store<STORE>::R* __restrict__ ib_g, int ib_cap) {
  lbm_body<Q, STORE, WALLS, MODE, IBB>(g, pl, u4, solid, bword, pose, posed, sp, tau, omega, guo0, rho0, red, forces,
                                       nodes, uprev, desc, cworld, ib_base, ib_word, ib_q, ib_g, ib_cap, blockIdx.x);
}

// One launch over the cells of many domains: block -> (domain, block of that domain's grid). Its
// plane pointers come from memory rather than the constant bank, so it gets more registers.
template <int Q, int STORE, bool WALLS, int MODE, bool IBB>
__global__ void __launch_bounds__(256, sizeof(typename Store<STORE>::R) == 8 ? 2 : 4) lbm_batched(const LbmArgs<Q, STORE>* __restrict__ args,
                                            const BlockMap* __restrict__ map) {
  const BlockMap m = map[blockIdx.x];
  const LbmArgs<Q, STORE>& a = args[m.domain];
  lbm_body<Q, STORE, WALLS, MODE, IBB>(a.g, a.pl, a.u4, a.solid, a.bword, a.pose, a.posed, a.sp, a.tau, a.omega,
                                       a.guo0, a.rho0, a.red, a.forces, nullptr, nullptr, nullptr, nullptr,
                                       nullptr, nullptr, nullptr, nullptr, 0, m.block);
}
#undef RWMI_LBM_BOUNDS

// ---- IBB links (Eq. 25) ahead of the LBM update ------------------------------------------
// Every fluid node of a flagged brick whose lattice neighbour x - e_i is a solid node owns the
// link (x, i). ibb_links_kernel gives every cell of a flagged brick its node word (bit 0: solid
// node; bit i: link i), appends a node's links in direction order (warp-aggregated) and keeps the
// index of its first one (or, when the list is full, an overflow slot); ibb_link_kernel then runs
// the 24-step binary32 bisection of every link and forms its G at full occupancy, instead of
// inside the update.
template <int Q, bool WALLS>
__global__ void __launch_bounds__(256) ibb_links_kernel(Geom g, const uint32_t* __restrict__ bword,
                                                        const uint16_t* __restrict__ nodes,
                                                        int32_t* __restrict__ base, uint32_t* __restrict__ word,
                                                        uint32_t* __restrict__ lcell,
                                                        uint32_t* __restrict__ lmeta, unsigned int* count, int cap,
                                                        int32_t* __restrict__ ocell, unsigned int* ocount, int ocap,
                                                        unsigned long long* __restrict__ status) {
  using L = Lat<Q>;
  // brick-major (as node_kernel): block 2 b + h takes half h of brick b; bricks that hold no
  // particle have no links and leave at once
  const uint32_t bq = blockIdx.x >> 1;
  if (!(bword[bq] >> 16)) return;   // block-uniform
  const uint32_t l = threadIdx.x + ((blockIdx.x & 1u) << 8);
  const uint32_t bi = bq % (uint32_t)g.nb[0], bj = (bq / (uint32_t)g.nb[0]) % (uint32_t)g.nb[1],
                 bk = bq / ((uint32_t)g.nb[0] * (uint32_t)g.nb[1]);
  uint32_t x = bi * BRICK + (l & 7u), y = bj * BRICK + ((l >> 3) & 7u), z = bk * BRICK + (l >> 6);
  const bool valid = x < (uint32_t)g.n[0] && y < (uint32_t)g.n[1] && z < (uint32_t)g.n[2];
  if (!valid) { x = 0; y = 0; z = 0; }   // outside the box (partial brick): no links
  const int c = (int)((z * (uint32_t)g.n[1] + y) * (uint32_t)g.n[0] + x);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int sy = nx, sz = (int)g.nxy;
  const int ox_p = x == 0 ? nx - 1 : -1, ox_m = (int)x == nx - 1 ? -(nx - 1) : 1;
  const int oy_p = y == 0 ? (ny - 1) * sy : -sy, oy_m = (int)y == ny - 1 ? -(ny - 1) * sy : sy;
  const int oz_p = z == 0 ? (nz - 1) * sz : -sz, oz_m = (int)z == nz - 1 ? -(nz - 1) * sz : sz;
  const bool wx_p = WALLS && g.wall[0] && x == 0, wx_m = WALLS && g.wall[0] && (int)x == nx - 1;
  const bool wy_p = WALLS && g.wall[1] && y == 0, wy_m = WALLS && g.wall[1] && (int)y == ny - 1;
  const bool wz_p = WALLS && g.wall[2] && z == 0, wz_m = WALLS && g.wall[2] && (int)z == nz - 1;
  auto off_of = [&](int i) {
    const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
    return (ex > 0 ? ox_p : ex < 0 ? ox_m : 0) + (ey > 0 ? oy_p : ey < 0 ? oy_m : 0) +
           (ez > 0 ? oz_p : ez < 0 ? oz_m : 0);
  };
  auto blocked = [&](int i) {
    const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
    return (ex > 0 && wx_p) || (ex < 0 && wx_m) || (ey > 0 && wy_p) || (ey < 0 && wy_m) ||
           (ez > 0 && wz_p) || (ez < 0 && wz_m);
  };
  unsigned lmask = 0u;
  if (valid) {
    const bool solid_node = nodes[c] != 0;
    if (!solid_node) {
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (!blocked(i) && nodes[c + off_of(i)] != 0) lmask |= 1u << i;
    }
    word[c] = lmask | (solid_node ? 1u : 0u);
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nl = __popc(lmask);
  int incl = nl;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(full, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(full, incl, 31);
  if (total == 0) return;   // warp-uniform
  unsigned first = 0;
  if (lane == 31) first = atomicAdd(count, (unsigned)total);
  first = __shfl_sync(full, first, 31) + (unsigned)(incl - nl);
  if (!nl) return;
  if (first + (unsigned)nl > (unsigned)cap) {   // the list is full: the cell takes an overflow slot
    for (unsigned k = first; k < (unsigned)cap && k < first + (unsigned)nl; ++k)
      lcell[k] = 0xffffffffu;   // its reserved list entries stay empty (ibb_link_kernel skips them)
    const unsigned slot = atomicAdd(ocount, 1u);
    if (slot < (unsigned)ocap) {
      ocell[slot] = c;
      base[c] = -1 - (int32_t)slot;
    } else {   // both full: this step's result is incomplete (rwmi_sync reports it)
      atomicAdd(&status[ST_IBB_OVERFLOW], 1ull);
      word[c] = 0u;   // the cell keeps its pulled populations
    }
    return;
  }
  base[c] = (int32_t)first;
  unsigned k = first;
  for (unsigned m = lmask; m; m &= m - 1u, ++k) {
    const int i = __ffs(m) - 1;
    lcell[k] = (uint32_t)c;
    lmeta[k] = (uint32_t)i | ((uint32_t)(nodes[c + off_of(i)] - 1) << 8);
  }
}

// One thread per listed link: q by the binary32 bisection (Eq. 25), then G_i (Eqs. 23-24) from
// the input populations and the previous velocity. The LBM kernel replaces the link's pulled
// population by G_i and, on the steps that read forces, forms the momentum exchange from q and G
// cell by cell in direction order.
template <int Q, int STORE, bool WALLS>
__global__ void __launch_bounds__(256) ibb_link_kernel(Geom g, const float4* __restrict__ cworld,
                                                       const ParticleDesc* __restrict__ desc,
                                                       const uint32_t* __restrict__ lcell,
                                                       const uint32_t* __restrict__ lmeta, const unsigned int* count,
                                                       unsigned int* count_next, int cap, float* __restrict__ qout,
                                                       typename Store<STORE>::R* __restrict__ gout,
                                                       const typename Store<STORE>::T* __restrict__ in0,
                                                       const float4* __restrict__ uprev,
                                                       const uint16_t* __restrict__ nodes,
                                                       const PoseF* __restrict__ pose, const PoseD* __restrict__ posed,
                                                       typename Store<STORE>::R rho0, const uint32_t* __restrict__ word,
                                                       const int32_t* __restrict__ ocell, const unsigned int* ocount,
                                                       unsigned int* ocount_next, int ocap) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using R = typename S::R;
  if (blockIdx.x == 0 && threadIdx.x == 0) {   // the next step appends there
    *count_next = 0u;
    *ocount_next = 0u;
  }
  const unsigned n = min(*count, (unsigned)cap);
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    if (lcell[j] == 0xffffffffu) continue;   // reserved by a cell that went to the overflow slots
    const int c = (int)lcell[j];
    const uint32_t meta = lmeta[j];
    const uint32_t z = fast_div((uint32_t)c, g.mxy, g.sxy), r = (uint32_t)c - z * g.nxy;
    const uint32_t y = fast_div(r, g.mx, g.sx), x = r - y * g.n[0];
    const int i = (int)(meta & 31u), p = (int)(meta >> 8), ip = L::opp(i);
    const float qv = ibb_link_q(cworld, desc[p].c0, desc[p].c1, (float)x + 0.5f, (float)y + 0.5f, (float)z + 0.5f,
                                L::e(ip, 0), L::e(ip, 1), L::e(ip, 2), g);
    qout[j] = qv;
    R sum = R(0);   // rho_f: x_f's own post-collision populations, summed in direction order
#pragma unroll
    for (int d = 0; d < Q; ++d) sum += S::ld(in0 + (size_t)d * g.ncell_pad + c);
    const R rho_f = S::shifted ? rho0 + sum : sum;
    const float4 u = uprev[c];
    const R uf[3] = {(R)u.x, (R)u.y, (R)u.z};
    R Gp, xw[3], uw[3];
    gout[j] = ibb_link_value<Q, STORE, WALLS>(g, in0, uprev, nodes, pose, posed, c, x, y, z, i, p, (R)qv, rho_f, uf,
                                              Gp, xw, uw);
  }
  // cells whose links did not fit in the list: all their links, by direction, in their slot of
  // the overflow table (cap + slot (Q - 1) + i - 1)
  const unsigned no = min(*ocount, (unsigned)ocap);
  for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < no; s += gridDim.x * blockDim.x) {
    const int c = ocell[s];
    const uint32_t z = fast_div((uint32_t)c, g.mxy, g.sxy), r = (uint32_t)c - z * g.nxy;
    const uint32_t y = fast_div(r, g.mx, g.sx), x = r - y * g.n[0];
    R sum = R(0);
    for (int d = 0; d < Q; ++d) sum += S::ld(in0 + (size_t)d * g.ncell_pad + c);
    const R rho_f = S::shifted ? rho0 + sum : sum;
    const float4 u = uprev[c];
    const R uf[3] = {(R)u.x, (R)u.y, (R)u.z};
    for (unsigned m = word[c] & ~1u; m; m &= m - 1u) {
      const int i = __ffs(m) - 1, ip = L::opp(i);
      int off = 0;
      pull_source<Q, WALLS>(g, x, y, z, i, off);
      const int p = (int)nodes[c + off] - 1;
      const float qv = ibb_link_q(cworld, desc[p].c0, desc[p].c1, (float)x + 0.5f, (float)y + 0.5f, (float)z + 0.5f,
                                  L::e(ip, 0), L::e(ip, 1), L::e(ip, 2), g);
      const size_t kk = (size_t)cap + (size_t)s * (Q - 1) + (size_t)(i - 1);
      qout[kk] = qv;
      R Gp, xw[3], uw[3];
      gout[kk] = ibb_link_value<Q, STORE, WALLS>(g, in0, uprev, nodes, pose, posed, c, x, y, z, i, p, (R)qv, rho_f,
                                                 uf, Gp, xw, uw);
    }
  }
}

void launch_ibb_links(int q, int storage, const Geom& g, BrickSet bs, const uint16_t* nodes, const IbbLinks& lk,
                      int par, const ParticleDesc* desc, const void* fin, const float* uprev, double rho0,
                      unsigned long long* status, int nsm, cudaStream_t st) {
  const bool walls = g.wall[0] || g.wall[1] || g.wall[2];
  const unsigned blocks = 2u * (unsigned)g.nb[0] * (unsigned)g.nb[1] * (unsigned)g.nb[2];   // two per brick
  unsigned int* cnt = lk.count + (par & 1);
  unsigned int* nxt = lk.count + ((par + 1) & 1);
  unsigned int* ocnt = lk.count + 2 + (par & 1);
  unsigned int* onxt = lk.count + 2 + ((par + 1) & 1);
  const float4* u4 = reinterpret_cast<const float4*>(uprev);
#define RWMI_IBB_LINKS(QQ, SS, WW)                                                                                   \
  do {                                                                                                             \
    using T_ = typename Store<SS>::T;                                                                              \
    using R_ = typename Store<SS>::R;                                                                              \
    ibb_links_kernel<QQ, WW><<<blocks, 256, 0, st>>>(g, bs.bword, nodes, lk.base, lk.word, lk.cell, lk.meta, cnt,   \
                                                      lk.cap, lk.ocell, ocnt, lk.ocap, status);                    \
    ibb_link_kernel<QQ, SS, WW><<<nsm * 8, 256, 0, st>>>(g, bs.cworld, desc, lk.cell, lk.meta, cnt, nxt, lk.cap,   \
                                                         lk.q, static_cast<R_*>(lk.g), static_cast<const T_*>(fin),\
                                                         u4, nodes, bs.pose, bs.posed, (R_)rho0, lk.word,          \
                                                         lk.ocell, ocnt, onxt, lk.ocap);                           \
  } while (0)
#define RWMI_IBB_W(QQ, SS) \
  if (walls) RWMI_IBB_LINKS(QQ, SS, true); else RWMI_IBB_LINKS(QQ, SS, false)
  // IBB is built for binary32-shifted and binary64-shifted storage
  if (q == 15) {
    if (storage == 3) { RWMI_IBB_W(15, 3); } else { RWMI_IBB_W(15, 1); }
  } else {
    if (storage == 3) { RWMI_IBB_W(19, 3); } else { RWMI_IBB_W(19, 1); }
  }
#undef RWMI_IBB_W
#undef RWMI_IBB_LINKS
}

template <int Q, int STORE, bool IBB>
static void launch_lbm_q(bool walls, bool reduce, const Geom& g, const void* fin, void* fout, float* u,
                         const uint16_t* solid, BrickSet bs, double tau, double rho0, double* red,
                         double* forces, cudaStream_t st, int bsz, const IbbArgs& ib, bool fused, bool update) {
  using T = typename Store<STORE>::T;
  using R = typename Store<STORE>::R;
  Planes<Q, T> pl;
  for (int i = 0; i < Q; ++i) {
    pl.in[i] = (const T*)fin + (size_t)i * g.ncell_pad;
    pl.out[i] = (T*)fout + (size_t)i * g.ncell_pad;
  }
  const int bsz_ok = (bsz == 64 || bsz == 128) ? bsz : 256;
  const dim3 grid((g.ncell + bsz_ok - 1) / bsz_ok), block(bsz_ok);
#define RWMI_LBM_ARGS g, pl, reinterpret_cast<float4*>(u), solid, bs.bword, bs.pose, bs.posed, bs.sp, (R)tau, (R)(1.0 / tau), (R)(1.0 - 0.5 / tau), (R)rho0, red, forces, ib.nodes, ib.uprev, ib.desc, bs.cworld, ib.base, ib.word, ib.q, static_cast<const R*>(ib.g), ib.cap
  if constexpr (STORE == 1 || STORE == 3) {   // the fused mode of free-DEM runs
    if (fused) {
      if (walls) lbm_kernel<Q, STORE, true, 2, IBB><<<grid, block, 0, st>>>(RWMI_LBM_ARGS);
      else lbm_kernel<Q, STORE, false, 2, IBB><<<grid, block, 0, st>>>(RWMI_LBM_ARGS);
      return;
    }
  }
  if (walls) {
    if (update) lbm_kernel<Q, STORE, true, 0, IBB><<<grid, block, 0, st>>>(RWMI_LBM_ARGS);
    if (reduce) lbm_kernel<Q, STORE, true, 1, IBB><<<grid, block, 0, st>>>(RWMI_LBM_ARGS);
  } else {
    if (update) lbm_kernel<Q, STORE, false, 0, IBB><<<grid, block, 0, st>>>(RWMI_LBM_ARGS);
    if (reduce) lbm_kernel<Q, STORE, false, 1, IBB><<<grid, block, 0, st>>>(RWMI_LBM_ARGS);
  }
#undef RWMI_LBM_ARGS
}

void launch_lbm(int q, int storage, bool reduce, const Geom& g, const void* fin, void* fout,
                float* u, const uint16_t* solid, BrickSet bs, double tau, double rho0, double* red,
                double* forces, unsigned long long* status, cudaStream_t st, int block, const IbbArgs* ibb,
                bool fused, bool update) {
  (void)status;
  const bool walls = g.wall[0] || g.wall[1] || g.wall[2];
  const IbbArgs none{};
  const IbbArgs& ib = ibb ? *ibb : none;
  // IBB is built for binary32-shifted and binary64 storage (the configuration check refuses the
  // others); the other storages run the partially saturated cells only
#define RWMI_LBM_PSM(QQ, SS) \
  launch_lbm_q<QQ, SS, false>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block, ib, fused, update)
#define RWMI_LBM_CASE(QQ, SS)                                                                           \
  if (ibb) launch_lbm_q<QQ, SS, true>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block, ib, fused, update); \
  else RWMI_LBM_PSM(QQ, SS)
  if (q == 15) {
    if (storage == 0) { RWMI_LBM_PSM(15, 0); }
    else if (storage == 1) { RWMI_LBM_CASE(15, 1); }
    else if (storage == 2) { RWMI_LBM_PSM(15, 2); }
    else { RWMI_LBM_CASE(15, 3); }
  } else {
    if (storage == 0) { RWMI_LBM_PSM(19, 0); }
    else if (storage == 1) { RWMI_LBM_CASE(19, 1); }
    else if (storage == 2) { RWMI_LBM_PSM(19, 2); }
    else { RWMI_LBM_CASE(19, 3); }
  }
#undef RWMI_LBM_CASE
#undef RWMI_LBM_PSM
}

// ---- TMA-staged update ------------------------------------------------------------------------
// The same update (MODE 0, partially saturated cells) with the pulls staged through shared
// memory: a resident grid walks the row tiles; per tile one thread issues Q tensor copies (one
// source row per direction, the rows at y - e_y, z - e_z wrapped on periodic axes) into one of
// TMA_STAGES buffers, completing on that buffer's mbarrier, TMA_STAGES - 1 tiles ahead of the
// compute. On a periodic x axis the halo element beyond the row's end is patched in from the other
// end; wall-blocked directions read their bounce-back population from global memory. Every wait
// is bounded: on expiry the kernel counts ST_TMA_TIMEOUT, waits (bounded) for its copies in
// flight and returns.
constexpr int TMA_STAGES = 3;
constexpr long long TMA_WAIT_CYCLES = 4000000000LL;   // about two seconds at the SM clock

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0u;
}
// Waits for the phase of parity `parity` to complete; false when `limit` cycles pass first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) return false;
  }
}

template <int Q, int STORE, bool WALLS>
__device__ __forceinline__ void tma_issue_tile(const CUtensorMap* map, typename Store<STORE>::T* stage, uint64_t* bar,
                                               const Geom& g, int tpr, int t, int stall_tile) {
  using L = Lat<Q>;
  using TR = TmaRow<STORE>;
  if (t == stall_tile) return;   // injected (rwmi_inject_wait_timeout): this tile's barrier never completes
  const int row = t / tpr, x0 = (t - row * tpr) * TMA_BX;
  const int ny = g.n[1], nz = g.n[2];
  const int y = row % ny, z = row / ny;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_addr(bar)), "r"((uint32_t)(Q * TR::bytes)) : "memory");
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int ey = L::e(i, 1), ez = L::e(i, 2);
    // periodic axes wrap; on a wall axis a blocked source row may fall outside (zero fill) and
    // is never read
    int ys = y - ey, zs = z - ez;
    if (!(WALLS && g.wall[1])) ys = ys < 0 ? ys + ny : ys >= ny ? ys - ny : ys;
    if (!(WALLS && g.wall[2])) zs = zs < 0 ? zs + nz : zs >= nz ? zs - nz : zs;
    const int rs = (ys < 0 || ys >= ny) ? -1 : zs * ny + ys;
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(smem_addr(stage + i * TR::pad)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x0 - TR::halo), "r"(rs),
           "r"(i), "r"(smem_addr(bar))
        : "memory");
  }
}

template <int Q, int STORE, bool WALLS>
__global__ void __launch_bounds__(TMA_BX, 8)
lbm_tma_kernel(const __grid_constant__ CUtensorMap tin, Geom g, Planes<Q, typename Store<STORE>::T> pl,
               float4* __restrict__ u4, const uint16_t* __restrict__ solid, const uint32_t* __restrict__ bword,
               const PoseF* __restrict__ pose, const PoseD* __restrict__ posed, const StepParams* __restrict__ sp,
               typename Store<STORE>::R tau, typename Store<STORE>::R omega, typename Store<STORE>::R guo0,
               typename Store<STORE>::R rho0, int tpr, unsigned long long* __restrict__ status, int stall_tile,
               long long wait_cycles) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  using T = typename S::T;
  using TR = TmaRow<STORE>;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) uint64_t bar[TMA_STAGES];
  // stage rows start on 128-byte boundaries (the launch adds 128 bytes of slack)
  T* stages = reinterpret_cast<T*>(tma_smem + ((128u - (smem_addr(tma_smem) & 127u)) & 127u));
  constexpr int stage_elems = Q * TR::pad;
  const int nx = g.n[0], ny = g.n[1];
  const int ntiles = ny * g.n[2] * tpr;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < TMA_STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < TMA_STAGES; ++s) {
      const int t = blockIdx.x + s * gridDim.x;
      if (t < ntiles) tma_issue_tile<Q, STORE, WALLS>(&tin, stages + s * stage_elems, &bar[s], g, tpr, t, stall_tile);
    }
  const bool xper = !(WALLS && g.wall[0]);
  int k = 0;
  bool expired = false;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int s = k % TMA_STAGES;
    const uint32_t parity = (uint32_t)(k / TMA_STAGES) & 1u;
    T* stage = stages + s * stage_elems;
    const bool ok = mbar_wait_bounded(&bar[s], parity, wait_cycles);
    if (__syncthreads_or(!ok)) { expired = true; break; }
    const int row = t / tpr, x0 = (t - row * tpr) * TMA_BX;
    const bool left = x0 == 0, right = x0 + TMA_BX >= nx;
    if (xper && (left || right)) {   // tile-uniform: patch the wrapped halo elements
      if (tid < Q) {
        const int i = tid, ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
        const int y = row % ny, z = row / ny;
        int ys = y - ey, zs = z - ez;
        const bool yw = WALLS && g.wall[1], zw = WALLS && g.wall[2];
        if (!yw) ys = ys < 0 ? ys + ny : ys >= ny ? ys - ny : ys;
        if (!zw) zs = zs < 0 ? zs + g.n[2] : zs >= g.n[2] ? zs - g.n[2] : zs;
        if (ys >= 0 && ys < ny && zs >= 0 && zs < g.n[2]) {
          const int rbase = (zs * ny + ys) * nx;
          if (left && ex > 0) stage[i * TR::pad + TR::halo - 1] = pl.in[i][rbase + nx - 1];
          if (right && ex < 0) stage[i * TR::pad + TR::halo + (nx - x0)] = pl.in[i][rbase];
        }
      }
      __syncthreads();
    }
    const bool valid = x0 + tid < nx;
    const int lx = valid ? tid : nx - 1 - x0;   // tail lanes recompute the row's last cell
    const uint32_t c = (uint32_t)row * (uint32_t)nx + (uint32_t)(x0 + lx);
    lbm_body<Q, STORE, WALLS, 0, false, true>(g, pl, u4, solid, bword, pose, posed, sp, tau, omega, guo0, rho0,
                                              nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                              nullptr, nullptr, 0, 0, stage, c, valid, lx);
    __syncthreads();   // every lane is done with this buffer
    if (tid == 0) {
      const int tn = t + TMA_STAGES * gridDim.x;
      if (tn < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the halo patch before new copies
        tma_issue_tile<Q, STORE, WALLS>(&tin, stage, &bar[s], g, tpr, tn, stall_tile);
      }
    }
  }
  if (expired) {   // count it; let the copies in flight land (bounded) before the block exits
    if (tid == 0) {
      atomicAdd(&status[ST_TMA_TIMEOUT], 1ull);
      for (int j = 0; j < TMA_STAGES; ++j) {
        const int kk = k + j, tt = blockIdx.x + kk * gridDim.x;
        if (tt < ntiles && tt != stall_tile)
          mbar_wait_bounded(&bar[kk % TMA_STAGES], (uint32_t)(kk / TMA_STAGES) & 1u, wait_cycles);
      }
    }
    __syncthreads();
  }
}

// Injected stalls (rwmi_inject_wait_timeout): the next n staged launches leave the copies of
// their first tile unissued and wait for them about a millisecond.
static std::atomic<int> g_tma_stalls{0};
int tma_inject_stalls(int n) { return g_tma_stalls.exchange(n < 0 ? 0 : n); }
static bool tma_take_stall() {
  int n = g_tma_stalls.load();
  while (n > 0 && !g_tma_stalls.compare_exchange_weak(n, n - 1)) {}
  return n > 0;
}

size_t lbm_tma_smem(int q, int storage) {
  const int pad_bytes = storage == 2 ? TmaRow<2>::pad * 2 : TmaRow<1>::pad * 4;
  return (size_t)TMA_STAGES * (size_t)q * (size_t)pad_bytes + 128;
}

bool lbm_tma_supported(int q, int storage, const Geom& g) {
  if (storage < 0 || storage > 2 || (q != 15 && q != 19)) return false;
  const int align = storage == 2 ? 8 : 4;   // row pitch a multiple of 16 bytes
  return g.n[0] % align == 0 && (int64_t)g.n[1] * g.n[2] < (1LL << 31);
}

// Tensor map of one population buffer: dims (x, row = y + ny z, direction), pitches nx and
// ncell_pad elements; box (TMA_BX + 2 halo, 1, 1); out-of-range elements read as zero.
bool lbm_tma_encode(int q, int storage, const Geom& g, const void* f, CUtensorMap* map) {
  if (!lbm_tma_supported(q, storage, g)) return false;
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) !=
            cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<Encode>(fn);
  }
  const int es = storage == 2 ? 2 : 4;
  const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1] * (cuuint64_t)g.n[2], (cuuint64_t)q};
  const cuuint64_t pitch[2] = {(cuuint64_t)g.n[0] * es, (cuuint64_t)g.ncell_pad * es};
  const cuuint32_t box[3] = {(cuuint32_t)(TMA_BX + 2 * (16 / es)), 1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, storage == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                            const_cast<void*>(f), dims, pitch, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int Q, int STORE>
static void launch_lbm_tma_q(bool walls, const CUtensorMap& map, const Geom& g, const void* fin, void* fout, float* u,
                             const uint16_t* solid, BrickSet bs, double tau, double rho0, unsigned long long* status,
                             int nsm, cudaStream_t st) {
  using T = typename Store<STORE>::T;
  using R = typename Store<STORE>::R;
  Planes<Q, T> pl;
  for (int i = 0; i < Q; ++i) {
    pl.in[i] = (const T*)fin + (size_t)i * g.ncell_pad;
    pl.out[i] = (T*)fout + (size_t)i * g.ncell_pad;
  }
  const int tpr = (g.n[0] + TMA_BX - 1) / TMA_BX;
  const size_t smem = lbm_tma_smem(Q, STORE);
  auto kern = walls ? lbm_tma_kernel<Q, STORE, true> : lbm_tma_kernel<Q, STORE, false>;
  static bool attr = false;   // per instantiation
  if (!attr) {
    cudaFuncSetAttribute(lbm_tma_kernel<Q, STORE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(lbm_tma_kernel<Q, STORE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  static int per_sm = 0;   // resident blocks per SM (shared memory bound)
  if (per_sm == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TMA_BX, smem);
  const int64_t ntiles = (int64_t)g.n[1] * g.n[2] * tpr;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)nsm * std::max(per_sm, 1));
  const bool stall = tma_take_stall();
  kern<<<grid, TMA_BX, smem, st>>>(map, g, pl, reinterpret_cast<float4*>(u), solid, bs.bword, bs.pose, bs.posed, bs.sp,
                                   (R)tau, (R)(1.0 / tau), (R)(1.0 - 0.5 / tau), (R)rho0, tpr, status,
                                   stall ? 0 : -1, stall ? 2000000LL : TMA_WAIT_CYCLES);
}

void launch_lbm_tma(int q, int storage, const CUtensorMap& map, const Geom& g, const void* fin, void* fout, float* u,
                    const uint16_t* solid, BrickSet bs, double tau, double rho0, unsigned long long* status, int nsm,
                    cudaStream_t st) {
  const bool walls = g.wall[0] || g.wall[1] || g.wall[2];
#define RWMI_TMA(QQ, SS) launch_lbm_tma_q<QQ, SS>(walls, map, g, fin, fout, u, solid, bs, tau, rho0, status, nsm, st)
  if (q == 15) {
    if (storage == 0) RWMI_TMA(15, 0); else if (storage == 1) RWMI_TMA(15, 1); else RWMI_TMA(15, 2);
  } else {
    if (storage == 0) RWMI_TMA(19, 0); else if (storage == 1) RWMI_TMA(19, 1); else RWMI_TMA(19, 2);
  }
#undef RWMI_TMA
}

template <int Q, int STORE>
static void fill_lbm_args(void* dst, const Geom& g, const void* fin, void* fout, float* u, const uint16_t* solid,
                          BrickSet bs, double tau, double rho0, double* red, double* forces) {
  using T = typename Store<STORE>::T;
  using R = typename Store<STORE>::R;
  LbmArgs<Q, STORE> a;
  a.g = g;
  for (int i = 0; i < Q; ++i) {
    a.pl.in[i] = (const T*)fin + (size_t)i * g.ncell_pad;
    a.pl.out[i] = (T*)fout + (size_t)i * g.ncell_pad;
  }
  a.u4 = reinterpret_cast<float4*>(u);
  a.solid = solid; a.bword = bs.bword; a.pose = bs.pose; a.posed = bs.posed; a.sp = bs.sp;
  a.tau = (R)tau; a.omega = (R)(1.0 / tau); a.guo0 = (R)(1.0 - 0.5 / tau); a.rho0 = (R)rho0;
  a.red = red; a.forces = forces;
  *static_cast<LbmArgs<Q, STORE>*>(dst) = a;
}

#define RWMI_LBM_STORAGES(QQ, M)                                        \
  (storage == 0 ? M(QQ, 0) : storage == 1 ? M(QQ, 1) : storage == 2 ? M(QQ, 2) : M(QQ, 3))
size_t lbm_args_size(int q, int storage) {
#define RWMI_SZ(QQ, SS) sizeof(LbmArgs<QQ, SS>)
  return q == 15 ? RWMI_LBM_STORAGES(15, RWMI_SZ) : RWMI_LBM_STORAGES(19, RWMI_SZ);
#undef RWMI_SZ
}
#undef RWMI_LBM_STORAGES

void lbm_args(void* dst, int q, int storage, const Geom& g, const void* fin, void* fout, float* u,
              const uint16_t* solid, BrickSet bs, double tau, double rho0, double* red, double* forces) {
#define RWMI_FILL(QQ, SS) fill_lbm_args<QQ, SS>(dst, g, fin, fout, u, solid, bs, tau, rho0, red, forces)
  if (q == 15) {
    if (storage == 0) RWMI_FILL(15, 0); else if (storage == 1) RWMI_FILL(15, 1);
    else if (storage == 2) RWMI_FILL(15, 2); else RWMI_FILL(15, 3);
  } else {
    if (storage == 0) RWMI_FILL(19, 0); else if (storage == 1) RWMI_FILL(19, 1);
    else if (storage == 2) RWMI_FILL(19, 2); else RWMI_FILL(19, 3);
  }
#undef RWMI_FILL
}

template <int Q, int STORE>
static void launch_lbm_batched_q(bool walls, int mode, const void* args, const BlockMap* map, int nblocks, int block,
                                 cudaStream_t st) {
  const LbmArgs<Q, STORE>* a = static_cast<const LbmArgs<Q, STORE>*>(args);
  if constexpr (STORE == 1 || STORE == 3) {   // the fused update and reduction
    if (mode == 2) {
      if (walls) lbm_batched<Q, STORE, true, 2, false><<<nblocks, block, 0, st>>>(a, map);
      else lbm_batched<Q, STORE, false, 2, false><<<nblocks, block, 0, st>>>(a, map);
      return;
    }
  }
  if (walls) {
    if (mode == 0) lbm_batched<Q, STORE, true, 0, false><<<nblocks, block, 0, st>>>(a, map);
    else lbm_batched<Q, STORE, true, 1, false><<<nblocks, block, 0, st>>>(a, map);
  } else {
    if (mode == 0) lbm_batched<Q, STORE, false, 0, false><<<nblocks, block, 0, st>>>(a, map);
    else lbm_batched<Q, STORE, false, 1, false><<<nblocks, block, 0, st>>>(a, map);
  }
}

void launch_lbm_batched(int q, int storage, bool walls, int mode, const void* args, const BlockMap* map,
                        int nblocks, int block, cudaStream_t st) {
  if (nblocks <= 0) return;
  block = (block == 64 || block == 128) ? block : 256;
#define RWMI_LB(QQ, SS) launch_lbm_batched_q<QQ, SS>(walls, mode, args, map, nblocks, block, st)
  if (q == 15) {
    if (storage == 0) RWMI_LB(15, 0); else if (storage == 1) RWMI_LB(15, 1);
    else if (storage == 2) RWMI_LB(15, 2); else RWMI_LB(15, 3);
  } else {
    if (storage == 0) RWMI_LB(19, 0); else if (storage == 1) RWMI_LB(19, 1);
    else if (storage == 2) RWMI_LB(19, 2); else RWMI_LB(19, 3);
  }
#undef RWMI_LB
}

}  // namespace rwmi
