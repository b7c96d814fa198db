// rwmi_lbm.cu -- the fused LBM step: pull stream (periodic wrap / half-way bounce-back) + BGK
// collide (Eqs. 12-15) with PSM solid coupling and Guo forcing; writes the populations, the
// velocity field and, on reduction steps, per-particle force/torque and the FP64 sums.
#include "rwmi_lattice.cuh"

namespace rwmi {

// ------------------------------------------------------------------------------------------
// Fused pull-stream + collide (Eqs. 12-15), partially saturated cells, Guo forcing.
// One thread per cell, flat index c = x + nx (y + ny z); direction planes are contiguous, so
// every pull load of a warp is one (shifted) coalesced row segment. Storage: binary32 f_i,
// binary32 f_i - w_i rho0 ("shifted") or binary16 shifted; arithmetic binary32.
// ------------------------------------------------------------------------------------------
// Base pointers of the Q direction planes (kernel parameters: constant-bank operands, so each
// access is one address multiply-add).
template <int Q, typename T> struct Planes {
  const T* in[Q];
  T* out[Q];
};

template <int Q, int STORE, bool WALLS, bool REDUCE>
__global__ void __launch_bounds__(256, 4) lbm_kernel(Geom g, Planes<Q, typename Store<STORE>::T> pl,
                                                  float4* __restrict__ u4,
                                                  const uint16_t* __restrict__ solid,
                                                  const uint32_t* __restrict__ bword,
                                                  const PoseF* __restrict__ pose,
                                                  const StepParams* __restrict__ sp, float tau,
                                                  float rho0, double* __restrict__ red,
                                                  double* __restrict__ forces) {
  using L = Lat<Q>;
  using S = Store<STORE>;
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = idx < g.ncell;
  const int c = (int)(valid ? idx : g.ncell - 1);   // tail lanes recompute the last cell, store nothing
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
  float f[Q];
  bool wall_cell = false;
  if (WALLS)
    wall_cell = (g.wall[0] && (x == 0 || (int)x == nx - 1)) || (g.wall[1] && (y == 0 || (int)y == ny - 1)) ||
                (g.wall[2] && (z == 0 || (int)z == nz - 1));
  if (!wall_cell) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
      const int off = (ex > 0 ? ox_p : ex < 0 ? ox_m : 0) + (ey > 0 ? oy_p : ey < 0 ? oy_m : 0) +
                      (ez > 0 ? oz_p : ez < 0 ? oz_m : 0);
      f[i] = S::ld(pl.in[i] + (c + off));
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
      const bool blk = (ex > 0 && bx_p) || (ex < 0 && bx_m) || (ey > 0 && by_p) || (ey < 0 && by_m) ||
                       (ez > 0 && bz_p) || (ez < 0 && bz_m);
      f[i] = blk ? S::ld(pl.in[L::opp(i)] + c) : S::ld(pl.in[i] + (c + off));
    }
  }
  // moments (Eqs. 14-15); with shifted storage f holds f_i - w_i rho0
  float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    drho += f[i];
    if (L::e(i, 0)) jx += L::e(i, 0) * f[i];
    if (L::e(i, 1)) jy += L::e(i, 1) * f[i];
    if (L::e(i, 2)) jz += L::e(i, 2) * f[i];
  }
  const float rho = S::shifted ? rho0 + drho : drho;
  const float Fx = sp->F[0], Fy = sp->F[1], Fz = sp->F[2];
  const float inv_rho = 1.0f / rho;
  const float ux = (jx + 0.5f * Fx) * inv_rho, uy = (jy + 0.5f * Fy) * inv_rho,
              uz = (jz + 0.5f * Fz) * inv_rho;
  const float uu = ux * ux + uy * uy + uz * uz;
  // partially saturated cell: solid word valid only in bricks flagged for this time
  float B = 0.0f, usx = 0.0f, usy = 0.0f, usz = 0.0f;
  int owner = -1;
  {
    const uint32_t b = ((z >> 3) * (uint32_t)g.nb[1] + (y >> 3)) * (uint32_t)g.nb[0] + (x >> 3);
    if (bword[b] >> 16) {
      const uint16_t sw = solid[c];
      const int cnt = sw & 0x7f;
      if (cnt && valid) {
        owner = sw >> 7;
        const float eps = (float)cnt * (1.0f / 64.0f);
        B = eps * (tau - 0.5f) / ((1.0f - eps) + (tau - 0.5f));
        const PoseF ps_ = pose[owner];
        float r[3] = {(float)x + 0.5f - ps_.o[0], (float)y + 0.5f - ps_.o[1], (float)z + 0.5f - ps_.o[2]};
        for (int a = 0; a < 3; ++a)
          if (!g.wall[a]) {
            const float na = (float)g.n[a];
            if (r[a] > 0.5f * na) r[a] -= na; else if (r[a] < -0.5f * na) r[a] += na;
          }
        usx = ps_.v[0] + ps_.w[1] * r[2] - ps_.w[2] * r[1];
        usy = ps_.v[1] + ps_.w[2] * r[0] - ps_.w[0] * r[2];
        usz = ps_.v[2] + ps_.w[0] * r[1] - ps_.w[1] * r[0];
      }
    }
  }
  const float omB = 1.0f - B;
  const float rtau = omB / tau;              // (1 - B) / tau
  const float guo = omB * (1.0f - 0.5f / tau);
  const float uF = ux * Fx + uy * Fy + uz * Fz;
  const float usus = usx * usx + usy * usy + usz * usz;
  float dpx = 0.0f, dpy = 0.0f, dpz = 0.0f;
  float out[Q];
  {  // rest direction; its own opposite: Omega_0 = feq_0(rho, u_s) - feq_0(rho, u)
    const float w = L::w(0);
    const float dev = -1.5f * uu;
    const float feq_s = S::shifted ? w * (drho + rho * dev) : w * rho * (1.0f + dev);
    const float om0 = B > 0.0f ? 1.5f * w * rho * (uu - usus) : 0.0f;
    out[0] = f[0] - rtau * (f[0] - feq_s) + guo * w * (-3.0f * uF) + B * om0;
  }
  // opposite pairs (i, i + H) share e.u
#pragma unroll
  for (int i = 1; i <= L::H; ++i) {
    const int io = i + L::H;
    const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
    const float w = L::w(i);
    const float eu = ex * ux + ey * uy + ez * uz;
    const float eF = ex * Fx + ey * Fy + ez * Fz;
    const float sym = 4.5f * eu * eu - 1.5f * uu;        // even part of feq / (w rho)
    const float base = S::shifted ? w * drho : w * rho;  // w rho (minus w rho0 when shifted)
    const float wr = w * rho;
    const float feq_p = base + wr * (3.0f * eu + sym);
    const float feq_m = base + wr * (-3.0f * eu + sym);
    const float gw = guo * w;
    out[i] = f[i] - rtau * (f[i] - feq_p) + gw * (3.0f * (eF - uF) + 9.0f * eu * eF);
    out[io] = f[io] - rtau * (f[io] - feq_m) + gw * (3.0f * (-eF - uF) + 9.0f * eu * eF);
    if (B > 0.0f) {
      const float eus = ex * usx + ey * usy + ez * usz;
      const float common = wr * (4.5f * (eus * eus - eu * eu) - 1.5f * (usus - uu));
      const float odd = wr * 3.0f * (eu + eus);
      const float om_p = (f[io] - f[i]) + odd + common;   // Omega_i
      const float om_m = (f[i] - f[io]) - odd + common;   // Omega_opp(i)
      out[i] += B * om_p;
      out[io] += B * om_m;
      const float dm = B * (om_p - om_m);                 // B (Omega_i e_i + Omega_opp e_opp) / e_i
      dpx += dm * ex; dpy += dm * ey; dpz += dm * ez;
    }
  }
  if (valid) {
#pragma unroll
    for (int i = 0; i < Q; ++i) S::st(pl.out[i] + c, out[i]);
    u4[c] = make_float4(ux, uy, uz, rho);
  }
  // hydrodynamic force on the owner particle: -B sum_i Omega_i e_i; torque about its origin
  const unsigned full = 0xffffffffu;
  const bool hasF = owner >= 0;
  if (__any_sync(full, hasF)) {
    float Fc[3] = {-dpx, -dpy, -dpz};
    float Tc[3] = {0.0f, 0.0f, 0.0f};
    if (hasF) {
      const PoseF ps_ = pose[owner];
      float r[3] = {(float)x + 0.5f - ps_.o[0], (float)y + 0.5f - ps_.o[1], (float)z + 0.5f - ps_.o[2]};
      for (int a = 0; a < 3; ++a)
        if (!g.wall[a]) {
          const float na = (float)g.n[a];
          if (r[a] > 0.5f * na) r[a] -= na; else if (r[a] < -0.5f * na) r[a] += na;
        }
      Tc[0] = r[1] * Fc[2] - r[2] * Fc[1];
      Tc[1] = r[2] * Fc[0] - r[0] * Fc[2];
      Tc[2] = r[0] * Fc[1] - r[1] * Fc[0];
    }
    const int key = hasF ? owner : -1;
    const int first = __shfl_sync(full, key, __ffs(__ballot_sync(full, hasF)) - 1);
    const bool uniform = __all_sync(full, !hasF || key == first);
    if (uniform) {
      float v[6] = {Fc[0], Fc[1], Fc[2], Tc[0], Tc[1], Tc[2]};
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        if (!hasF) v[m] = 0.0f;
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
  if (REDUCE) {   // sums of (rho - rho0) and sum_i f_i e_i (pre-collision): binary32 within the
                  // block (256 small deviations), FP64 across blocks (GB300's FP64 pipe is narrow)
    float v[4] = {valid ? (S::shifted ? drho : rho - rho0) : 0.0f, valid ? jx : 0.0f,
                  valid ? jy : 0.0f, valid ? jz : 0.0f};
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(full, v[m], o);
    __shared__ float s_red[8][4];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
      for (int m = 0; m < 4; ++m) s_red[wid][m] = v[m];
    __syncthreads();
    if (threadIdx.x < 4) {   // striped slots keep the FP64 atomics of 65536 blocks uncontended
      float s = 0.0f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_red[w][threadIdx.x];
      atomicAdd(&red[4 * (blockIdx.x % RED_SLOTS) + threadIdx.x], (double)s);
    }
  }
}

template <int Q, int STORE>
static void launch_lbm_q(bool walls, bool reduce, const Geom& g, const void* fin, void* fout, float* u,
                         const uint16_t* solid, BrickSet bs, float tau, float rho0, double* red,
                         double* forces, cudaStream_t st, int bsz) {
  using T = typename Store<STORE>::T;
  Planes<Q, T> pl;
  for (int i = 0; i < Q; ++i) {
    pl.in[i] = (const T*)fin + (size_t)i * g.ncell_pad;
    pl.out[i] = (T*)fout + (size_t)i * g.ncell_pad;
  }
  float4* u4 = reinterpret_cast<float4*>(u);
  const int bsz_ok = (bsz == 64 || bsz == 128) ? bsz : 256;
  const dim3 grid((g.ncell + bsz_ok - 1) / bsz_ok), block(bsz_ok);
  if (walls) {
    if (reduce) lbm_kernel<Q, STORE, true, true><<<grid, block, 0, st>>>(g, pl, u4, solid, bs.bword, bs.pose, bs.sp, tau, rho0, red, forces);
    else lbm_kernel<Q, STORE, true, false><<<grid, block, 0, st>>>(g, pl, u4, solid, bs.bword, bs.pose, bs.sp, tau, rho0, red, forces);
  } else {
    if (reduce) lbm_kernel<Q, STORE, false, true><<<grid, block, 0, st>>>(g, pl, u4, solid, bs.bword, bs.pose, bs.sp, tau, rho0, red, forces);
    else lbm_kernel<Q, STORE, false, false><<<grid, block, 0, st>>>(g, pl, u4, solid, bs.bword, bs.pose, bs.sp, tau, rho0, red, forces);
  }
}

void launch_lbm(int q, int storage, bool reduce, const Geom& g, const void* fin, void* fout,
                float* u, const uint16_t* solid, BrickSet bs, float tau, float rho0, double* red,
                double* forces, unsigned long long* status, cudaStream_t st, int block) {
  (void)status;
  const bool walls = g.wall[0] || g.wall[1] || g.wall[2];
  if (q == 15) {
    if (storage == 0) launch_lbm_q<15, 0>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block);
    else if (storage == 1) launch_lbm_q<15, 1>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block);
    else launch_lbm_q<15, 2>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block);
  } else {
    if (storage == 0) launch_lbm_q<19, 0>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block);
    else if (storage == 1) launch_lbm_q<19, 1>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block);
    else launch_lbm_q<19, 2>(walls, reduce, g, fin, fout, u, solid, bs, tau, rho0, red, forces, st, block);
  }
}

}  // namespace rwmi
