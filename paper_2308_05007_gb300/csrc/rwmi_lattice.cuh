// rwmi_lattice.cuh -- velocity sets and population storage policies shared by the LBM kernel
// and the initialisation / read-back kernels.
#pragma once
#include <cuda_fp16.h>

#include "rwmi_internal.cuh"

namespace rwmi {

// ------------------------------------------------------------------------------------------
// Velocity sets. Directions 1..H form one half of the set; direction i + H is the opposite of i.
//   D3Q15 half: (1,0,0) (0,1,0) (0,0,1) (1,1,1) (1,1,-1) (1,-1,1) (1,-1,-1)
//   D3Q19 half: (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)
// Weights: D3Q15 2/9, 1/9, 1/72; D3Q19 1/3, 1/18, 1/36 (c_s^2 = 1/3).
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr int half15(int i, int a) {
  return a == 0 ? (i == 2 || i == 3 ? 0 : 1)
       : a == 1 ? (i == 1 || i == 3 ? 0 : (i == 2 || i == 4 || i == 5) ? 1 : -1)
                : (i == 1 || i == 2 ? 0 : (i == 3 || i == 4 || i == 6) ? 1 : -1);
}
__host__ __device__ constexpr int half19(int i, int a) {
  return a == 0 ? ((i == 1 || (i >= 4 && i <= 7)) ? 1 : 0)
       : a == 1 ? ((i == 2 || i == 4 || i == 8 || i == 9) ? 1 : (i == 5 ? -1 : 0))
                : ((i == 3 || i == 6 || i == 8) ? 1 : ((i == 7 || i == 9) ? -1 : 0));
}
template <int Q> struct Lat {
  static constexpr int H = (Q - 1) / 2;
  __host__ __device__ static constexpr int e(int i, int a) {
    return i == 0 ? 0
         : i <= H ? (Q == 15 ? half15(i, a) : half19(i, a))
                  : -(Q == 15 ? half15(i - H, a) : half19(i - H, a));
  }
  __host__ __device__ static constexpr int e2(int i) {
    return e(i, 0) * e(i, 0) + e(i, 1) * e(i, 1) + e(i, 2) * e(i, 2);
  }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= H ? i + H : i - H); }
  // weight in the arithmetic type R (each a correctly rounded constant)
  template <typename R> __host__ __device__ static constexpr R wt(int i) {
    return Q == 15 ? (e2(i) == 0 ? R(2) / R(9) : e2(i) == 1 ? R(1) / R(9) : R(1) / R(72))
                   : (e2(i) == 0 ? R(1) / R(3) : e2(i) == 1 ? R(1) / R(18) : R(1) / R(36));
  }
};


// Population storage: binary32 f_i, binary32 f_i - w_i rho0 ("shifted"), binary16 shifted (all
// with binary32 arithmetic), or binary64 shifted with binary64 arithmetic.
template <int STORE> struct Store;
template <> struct Store<0> {   // binary32 f_i
  using T = float;
  using R = float;              // arithmetic type of the LBM update
  static constexpr bool shifted = false;
  __device__ static R ld(const T* p) { return *p; }
  __device__ static void st(T* p, R v) { *p = v; }
};
template <> struct Store<1> {   // binary32 f_i - w_i rho0
  using T = float;
  using R = float;
  static constexpr bool shifted = true;
  __device__ static R ld(const T* p) { return *p; }
  __device__ static void st(T* p, R v) { *p = v; }
};
template <> struct Store<2> {   // binary16 f_i - w_i rho0, binary32 arithmetic
  using T = __half;
  using R = float;
  static constexpr bool shifted = true;
  __device__ static R ld(const T* p) { return __half2float(*p); }
  __device__ static void st(T* p, R v) { *p = __float2half_rn(v); }
};
template <> struct Store<3> {   // binary64 f_i - w_i rho0, binary64 arithmetic (reference run)
  using T = double;
  using R = double;
  static constexpr bool shifted = true;
  __device__ static R ld(const T* p) { return *p; }
  __device__ static void st(T* p, R v) { *p = v; }
};

// Pose of particle p in the arithmetic type: the binary64 copy for the binary64 update.
template <typename R>
__device__ __forceinline__ void load_pose(const PoseF* pose, const PoseD* posed, int p, R* o, R* v, R* w) {
  if (sizeof(R) == 8) {
    const PoseD& q = posed[p];
    for (int a = 0; a < 3; ++a) { o[a] = (R)q.o[a]; v[a] = (R)q.v[a]; w[a] = (R)q.w[a]; }
  } else {
    const PoseF q = pose[p];
    for (int a = 0; a < 3; ++a) { o[a] = (R)q.o[a]; v[a] = (R)q.v[a]; w[a] = (R)q.w[a]; }
  }
}

// Rigid velocity v_p + omega_p x (x - o_p) of particle p at the point (x, y, z), minimum image.
template <typename R>
__device__ __forceinline__ void rigid_velocity(const Geom& g, const PoseF* pose, const PoseD* posed, int p,
                                               R x, R y, R z, R* u) {
  R po[3], pv[3], pw[3];
  load_pose<R>(pose, posed, p, po, pv, pw);
  R r[3] = {x - po[0], y - po[1], z - po[2]};
  for (int a = 0; a < 3; ++a)
    if (!g.wall[a]) {
      const R na = (R)g.n[a];
      if (r[a] > R(0.5) * na) r[a] -= na; else if (r[a] < -R(0.5) * na) r[a] += na;
    }
  u[0] = pv[0] + pw[1] * r[2] - pw[2] * r[1];
  u[1] = pv[1] + pw[2] * r[0] - pw[0] * r[2];
  u[2] = pv[2] + pw[0] * r[1] - pw[1] * r[0];
}

}  // namespace rwmi
