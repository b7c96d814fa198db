// rwmi_dem.cu -- free DEM of the metaball particles (Section 2.2, Eqs. 4-11): sphero-metaball
// contact geometry, linear spring-dashpot normal force, the Eq. 5 tangential spring with its
// Coulomb limit, and the Eq. 4 integration.
//
// This translation unit is built without FMA contraction (-fmad=false) and takes IEEE division
// and square roots, so every binary64 operation rounds exactly as written. With the fluid force
// switched off the trajectories then follow the CPU oracle's bit for bit, which the GPU tests
// check; the formulas and their readings are the oracle's.
//
// One DEM step is two launches (or, for up to 128 particles, every DEM step of an LBM step is one
// single-block launch, dem_fused_kernel, with block barriers between the two phases):
//   dem_contacts_kernel   one thread per pair slot (i < j) and per wall slot (particle, face):
//                         reach test, Newton-Raphson geometry, force law; writes the slot's
//                         force and torques (zero when apart) and its spring and Newton point;
//   dem_integrate_kernel  one thread per particle: sums its slots in a fixed order (pairs by
//                         partner index, then faces), adds the fluid force and gravity, advances
//                         velocity, origin, spin and orientation.
// Kernels wait on nothing; the launches follow each other on one stream.
#include "rwmi_internal.cuh"

namespace rwmi {
namespace {

constexpr int NEWTON_NEW = 24;        // Newton iterations (at most) from the deterministic start
constexpr int NEWTON_CONT = 6;        // ... from the previous DEM step's point (pair within reach then)
constexpr int SURFACE_ITERS = 24;     // bracketed Newton iterations for Eq. 8's q
constexpr int SURFACE_HALVINGS = 16;  // halvings of the first-order q looking for an inside point

__device__ void quat_matrix(const double* q, double R[3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1.0 - 2.0 * (y * y + z * z);
  R[0][1] = 2.0 * (x * y - w * z);
  R[0][2] = 2.0 * (x * z + w * y);
  R[1][0] = 2.0 * (x * y + w * z);
  R[1][1] = 1.0 - 2.0 * (x * x + z * z);
  R[1][2] = 2.0 * (y * z - w * x);
  R[2][0] = 2.0 * (x * z - w * y);
  R[2][1] = 2.0 * (y * z + w * x);
  R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

// Internal (zoomed) control points of particle p about origin org: positions and weights
__device__ int internal_points(const DemArgs& a, int p, const double org[3], double* cw, double* kw) {
  double R[3][3];
  quat_matrix(a.st + 13 * p + 3, R);
  const double s = a.zoom[p];
  const ParticleDesc& d = a.desc[p];
  int n = 0;
  for (int i = d.c0; i < d.c1 && n < DEM_MAX_CP; ++i, ++n) {
    const float4 cb = a.cbody[i];
    const double b[3] = {s * (double)cb.x, s * (double)cb.y, s * (double)cb.z};
    for (int e = 0; e < 3; ++e) cw[3 * n + e] = org[e] + R[e][0] * b[0] + R[e][1] * b[1] + R[e][2] * b[2];
    kw[n] = s * s * (double)cb.w;
  }
  return n;
}

// Eq. 3 with gradient and Hessian (xx yy zz xy xz yz) at x
__device__ double mb_eval(const double* cw, const double* kw, int n, const double x[3], double g[3], double H[6]) {
  double f = 0.0;
  for (int e = 0; e < 3; ++e) g[e] = 0.0;
  for (int m = 0; m < 6; ++m) H[m] = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r[3] = {x[0] - cw[3 * i], x[1] - cw[3 * i + 1], x[2] - cw[3 * i + 2]};
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double inv2 = 1.0 / r2, k = kw[i];
    const double fi = k * inv2;
    f += fi;
    const double c1 = -2.0 * fi * inv2;
    const double c2 = 8.0 * fi * inv2 * inv2;
    for (int e = 0; e < 3; ++e) g[e] += c1 * r[e];
    H[0] += c1 + c2 * r[0] * r[0];
    H[1] += c1 + c2 * r[1] * r[1];
    H[2] += c1 + c2 * r[2] * r[2];
    H[3] += c2 * r[0] * r[1];
    H[4] += c2 * r[0] * r[2];
    H[5] += c2 * r[1] * r[2];
  }
  return f;
}

__device__ bool solve3(const double A[3][3], const double b[3], double d[3]) {
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
                   - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                   + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(fabs(det) > 1e-300)) return false;
  d[0] = (b[0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (b[1] * A[2][2] - A[1][2] * b[2])
          + A[0][2] * (b[1] * A[2][1] - A[1][1] * b[2])) / det;
  d[1] = (A[0][0] * (b[1] * A[2][2] - A[1][2] * b[2]) - b[0] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
          + A[0][2] * (A[1][0] * b[2] - b[1] * A[2][0])) / det;
  d[2] = (A[0][0] * (A[1][1] * b[2] - b[1] * A[2][1]) - A[0][1] * (A[1][0] * b[2] - b[1] * A[2][0])
          + b[0] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / det;
  return true;
}

// Newton step, at most one lattice unit long; false when singular or converged (step < 1e-12)
__device__ bool newton_update(const double A[3][3], const double G[3], double x[3]) {
  const double b[3] = {-G[0], -G[1], -G[2]};
  double d[3];
  if (!solve3(A, b, d)) return false;
  const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double sc = len > 1.0 ? 1.0 / len : 1.0;
  for (int e = 0; e < 3; ++e) x[e] += sc * d[e];
  return len > 1e-12;
}

// Eq. 8: x_c = x_m + q grad f(x_m) with f(x_c) = 1, the crossing nearest to x_m (first-order
// Taylor q, bracket by halving to an inside point, bracketed Newton in q)
__device__ void surface_along(const double* c, const double* k, int n, const double xm[3], double xc[3]) {
  double g[3], gx[3], H[6], x[3];
  const double f = mb_eval(c, k, n, xm, g, H);
  const double q1 = (1.0 - f) / (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double lo = 0.0, hi = q1, q = q1;
  bool inside = false;
  for (int h = 0; h <= SURFACE_HALVINGS; ++h) {
    for (int e = 0; e < 3; ++e) x[e] = xm[e] + hi * g[e];
    if (mb_eval(c, k, n, x, gx, H) >= 1.0) { inside = true; break; }
    hi = 0.5 * hi;
  }
  if (inside) {
    q = hi;
    for (int it = 0; it < SURFACE_ITERS; ++it) {
      for (int e = 0; e < 3; ++e) x[e] = xm[e] + q * g[e];
      const double fx = mb_eval(c, k, n, x, gx, H);
      if (fx == 1.0) break;
      if (fx > 1.0) hi = q; else lo = q;
      const double dq = gx[0] * g[0] + gx[1] * g[1] + gx[2] * g[2];
      double qn = fabs(dq) > 1e-300 ? q - (fx - 1.0) / dq : 0.5 * (lo + hi);
      if (!(qn > lo && qn < hi)) qn = 0.5 * (lo + hi);
      if (qn == q) break;
      q = qn;
    }
  }
  for (int e = 0; e < 3; ++e) xc[e] = xm[e] + q * g[e];
}

// Eqs. 7-9 for one pair; xm: start (cont) and result. Returns delta; writes n (0 -> 1), x_cp.
__device__ double pair_geom(const double* c0, const double* k0, int n0, const double* c1, const double* k1, int n1,
                            double Rs0, double Rs1, bool cont, double xm[3], double nrm[3], double xcp[3]) {
  if (!cont) {
    int ba = 0, bb = 0;
    double best = INFINITY;
    for (int a = 0; a < n0; ++a)
      for (int b = 0; b < n1; ++b) {
        const double d[3] = {c1[3 * b] - c0[3 * a], c1[3 * b + 1] - c0[3 * a + 1], c1[3 * b + 2] - c0[3 * a + 2]};
        const double gap = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - sqrt(k0[a]) - sqrt(k1[b]);
        if (gap < best) { best = gap; ba = a; bb = b; }
      }
    const double ra = sqrt(k0[ba]), rb = sqrt(k1[bb]), w = ra / (ra + rb);
    for (int e = 0; e < 3; ++e) xm[e] = c0[3 * ba + e] + w * (c1[3 * bb + e] - c0[3 * ba + e]);
  }
  const int iters = cont ? NEWTON_CONT : NEWTON_NEW;
  for (int it = 0; it < iters; ++it) {
    double g0[3], g1[3], H0[6], H1[6];
    mb_eval(c0, k0, n0, xm, g0, H0);
    mb_eval(c1, k1, n1, xm, g1, H1);
    const double G[3] = {g0[0] + g1[0], g0[1] + g1[1], g0[2] + g1[2]};
    const double A[3][3] = {{H0[0] + H1[0], H0[3] + H1[3], H0[4] + H1[4]},
                            {H0[3] + H1[3], H0[1] + H1[1], H0[5] + H1[5]},
                            {H0[4] + H1[4], H0[5] + H1[5], H0[2] + H1[2]}};
    if (!newton_update(A, G, xm)) break;
  }
  double xc0[3], xc1[3];
  surface_along(c0, k0, n0, xm, xc0);
  surface_along(c1, k1, n1, xm, xc1);
  const double d[3] = {xc1[0] - xc0[0], xc1[1] - xc0[1], xc1[2] - xc0[2]};
  const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const double delta = Rs0 + Rs1 - dist;
  for (int e = 0; e < 3; ++e) nrm[e] = dist > 0.0 ? d[e] / dist : 0.0;
  for (int e = 0; e < 3; ++e) xcp[e] = xc0[e] + (Rs0 - 0.5 * delta) * nrm[e];
  return delta;
}

// Eqs. 10-11 for the face `side` of walled axis ax at 0 or L; n into the box
__device__ double wall_geom(const double* c, const double* k, int n, int ax, int side, double L, double Rs, bool cont,
                            double xm[3], double nrm[3], double xcp[3]) {
  const double sg = side ? -1.0 : 1.0;
  if (!cont) {
    int bi = 0;
    double best = INFINITY;
    for (int i = 0; i < n; ++i) {
      const double reach = side ? -(c[3 * i + ax] + sqrt(k[i])) : c[3 * i + ax] - sqrt(k[i]);
      if (reach < best) { best = reach; bi = i; }
    }
    for (int e = 0; e < 3; ++e) xm[e] = c[3 * bi + e];
    xm[ax] -= sg * sqrt(k[bi]);
  }
  int b = (ax + 1) % 3, cc = (ax + 2) % 3;
  if (b > cc) { const int t = b; b = cc; cc = t; }
  const int iters = cont ? NEWTON_CONT : NEWTON_NEW;
  for (int it = 0; it < iters; ++it) {
    double g[3], H6[6];
    const double f = mb_eval(c, k, n, xm, g, H6);
    const double H[3][3] = {{H6[0], H6[3], H6[4]}, {H6[3], H6[1], H6[5]}, {H6[4], H6[5], H6[2]}};
    const double G[3] = {g[b], g[cc], f - 1.0};
    const double A[3][3] = {{H[b][0], H[b][1], H[b][2]}, {H[cc][0], H[cc][1], H[cc][2]}, {g[0], g[1], g[2]}};
    if (!newton_update(A, G, xm)) break;
  }
  double xcw[3];
  for (int e = 0; e < 3; ++e) { xcw[e] = xm[e]; nrm[e] = 0.0; }
  xcw[ax] = side ? L : 0.0;
  nrm[ax] = sg;
  const double dist = (xm[ax] - xcw[ax]) * sg;
  const double delta = Rs - dist;
  for (int e = 0; e < 3; ++e) xcp[e] = xcw[e] + 0.5 * delta * nrm[e];
  return delta;
}

__device__ void point_velocity(const DemArgs& a, int p, const double org[3], const double x[3], double v[3]) {
  const double* st = a.st + 13 * p;
  const double r[3] = {x[0] - org[0], x[1] - org[1], x[2] - org[2]};
  const double* w = st + 10;
  v[0] = st[7] + (w[1] * r[2] - w[2] * r[1]);
  v[1] = st[8] + (w[2] * r[0] - w[0] * r[2]);
  v[2] = st[9] + (w[0] * r[1] - w[1] * r[0]);
}

// Normal spring-dashpot and Eq. 5 on body i; n from i towards the other body
__device__ void contact_force(const DemArgs& a, double delta, const double n[3], const double vi[3],
                              const double vj[3], double* xi, double F[3]) {
  const double vr[3] = {vj[0] - vi[0], vj[1] - vi[1], vj[2] - vi[2]};
  const double vn = vr[0] * n[0] + vr[1] * n[1] + vr[2] * n[2];
  double Fn = a.kn * delta - a.etan * vn;
  if (Fn < 0.0) Fn = 0.0;
  const double vt[3] = {vr[0] - vn * n[0], vr[1] - vn * n[1], vr[2] - vn * n[2]};
  const double xn = xi[0] * n[0] + xi[1] * n[1] + xi[2] * n[2];
  for (int e = 0; e < 3; ++e) xi[e] = (xi[e] - xn * n[e]) + vt[e] * a.dt;
  double Ft[3];
  for (int e = 0; e < 3; ++e) Ft[e] = a.kt * xi[e] + a.etat * vt[e];
  const double mag = sqrt(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
  const double lim = a.mus * Fn;
  if (mag > lim) {
    const double sc = lim / mag;
    for (int e = 0; e < 3; ++e) {
      Ft[e] = Ft[e] * sc;
      xi[e] = a.kt > 0.0 ? (Ft[e] - a.etat * vt[e]) / a.kt : 0.0;
    }
  }
  for (int e = 0; e < 3; ++e) F[e] = Ft[e] - Fn * n[e];
}

__device__ void cross3(const double u[3], const double v[3], double w[3]) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

__device__ void clear3(double* v) { v[0] = v[1] = v[2] = 0.0; }

// One pair slot (i < j)
__device__ void pair_slot(const DemArgs& a, int i, int j) {
  const size_t pr = (size_t)i * a.P + j;
  double* F = a.pF + 3 * pr;
  double* Ti = a.pTi + 3 * pr;
  double* Tj = a.pTj + 3 * pr;
  double* xi = a.xi + 3 * pr;
  {   // binary32 reach prefilter: bound spheres apart by more than a margin cannot touch
    const float4 pi = a.posf[i], pj = a.posf[j];
    const float dv[3] = {pj.x - pi.x, pj.y - pi.y, pj.z - pi.z};
    float d2 = 0.0f;
    for (int e = 0; e < 3; ++e) {
      float dd = dv[e];
      if (!a.wall[e]) dd -= (float)a.n[e] * rintf(dd / (float)a.n[e]);
      d2 += dd * dd;
    }
    const float reach = pi.w + pj.w + 0.01f;
    if (d2 > reach * reach) {   // the slot's forces are read only while in contact
      if (a.act[pr]) { a.act[pr] = 0; clear3(xi); }
      return;
    }
  }
  clear3(F); clear3(Ti); clear3(Tj);
  const double* si = a.st + 13 * i;
  const double* sj = a.st + 13 * j;
  double oj[3];
  for (int e = 0; e < 3; ++e) {   // minimum image of j's origin seen from i's
    double d = sj[e] - si[e];
    if (!a.wall[e]) d -= (double)a.n[e] * floor(d / (double)a.n[e] + 0.5);
    oj[e] = si[e] + d;
  }
  const double d[3] = {oj[0] - si[0], oj[1] - si[1], oj[2] - si[2]};
  const double reach = (double)a.desc[i].rb + (double)a.desc[j].rb;
  if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= reach * reach) {
    a.act[pr] = 0;
    clear3(xi);
    return;
  }
  double c0[3 * DEM_MAX_CP], k0[DEM_MAX_CP], c1[3 * DEM_MAX_CP], k1[DEM_MAX_CP];
  const int n0 = internal_points(a, i, si, c0, k0);
  const int n1 = internal_points(a, j, oj, c1, k1);
  double nrm[3], xcp[3];
  double xm[3] = {a.xm[3 * pr], a.xm[3 * pr + 1], a.xm[3 * pr + 2]};
  const double delta = pair_geom(c0, k0, n0, c1, k1, n1, a.Rs[i], a.Rs[j], a.act[pr] != 0, xm, nrm, xcp);
  for (int e = 0; e < 3; ++e) a.xm[3 * pr + e] = xm[e];
  if (!(delta > 0.0)) {
    a.act[pr] = 0;
    clear3(xi);
    return;
  }
  a.act[pr] = 1;
  double vi[3], vj[3];
  point_velocity(a, i, si, xcp, vi);
  point_velocity(a, j, oj, xcp, vj);
  contact_force(a, delta, nrm, vi, vj, xi, F);
  const double ri[3] = {xcp[0] - si[0], xcp[1] - si[1], xcp[2] - si[2]};
  const double rj[3] = {xcp[0] - oj[0], xcp[1] - oj[1], xcp[2] - oj[2]};
  const double Fj[3] = {-F[0], -F[1], -F[2]};
  cross3(ri, F, Ti);
  cross3(rj, Fj, Tj);
}

// One wall slot: particle p, face f = 2 axis + side
__device__ void wall_slot(const DemArgs& a, int p, int f) {
  const size_t wi = 6 * (size_t)p + f;
  const int ax = f >> 1, side = f & 1;
  double* F = a.wF + 3 * wi;
  double* T = a.wT + 3 * wi;
  double* xi = a.xiw + 3 * wi;
  {   // binary32 reach prefilter
    const float4 pf = a.posf[p];
    const float c = ax == 0 ? pf.x : ax == 1 ? pf.y : pf.z;
    const float gapf = side ? (float)a.n[ax] - c : c;
    if (!a.wall[ax] || gapf > pf.w + 0.01f) {
      if (a.actw[wi]) { a.actw[wi] = 0; clear3(xi); }
      return;
    }
  }
  clear3(F); clear3(T);
  const double* sp = a.st + 13 * p;
  const double L = (double)a.n[ax];
  const double gap = side ? L - sp[ax] : sp[ax];
  if (!a.wall[ax] || gap >= (double)a.desc[p].rb) {
    a.actw[wi] = 0;
    clear3(xi);
    return;
  }
  double c[3 * DEM_MAX_CP], k[DEM_MAX_CP];
  const int n = internal_points(a, p, sp, c, k);
  double nrm[3], xcp[3];
  double xm[3] = {a.xmw[3 * wi], a.xmw[3 * wi + 1], a.xmw[3 * wi + 2]};
  const double delta = wall_geom(c, k, n, ax, side, L, a.Rs[p], a.actw[wi] != 0, xm, nrm, xcp);
  for (int e = 0; e < 3; ++e) a.xmw[3 * wi + e] = xm[e];
  if (!(delta > 0.0)) {
    a.actw[wi] = 0;
    clear3(xi);
    return;
  }
  a.actw[wi] = 1;
  double vi[3];
  const double vw[3] = {0.0, 0.0, 0.0};
  point_velocity(a, p, sp, xcp, vi);
  const double nw[3] = {-nrm[0], -nrm[1], -nrm[2]};
  contact_force(a, delta, nw, vi, vw, xi, F);
  const double r[3] = {xcp[0] - sp[0], xcp[1] - sp[1], xcp[2] - sp[2]};
  cross3(r, F, T);
}

__global__ void __launch_bounds__(64) dem_contacts_kernel(DemArgs a, int npairs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < npairs) {
    int i = 0, rem = k;   // slot k -> pair (i, j), rows of P - 1 - i entries
    while (rem >= a.P - 1 - i) { rem -= a.P - 1 - i; ++i; }
    pair_slot(a, i, i + 1 + rem);
  } else if (k < npairs + 6 * a.P) {
    const int w = k - npairs;
    wall_slot(a, w / 6, w % 6);
  }
}

__device__ void integrate_particle(const DemArgs& a, int p);

__global__ void dem_integrate_kernel(DemArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < a.P) integrate_particle(a, p);
}

// Every DEM step of one LBM step in one block: contact slots, a block barrier, integration, a
// block barrier. For small particle counts, where launch latency would dominate.
constexpr int DEM_FUSED_THREADS = 512;
constexpr int DEM_FUSED_MAX_P = 128;
__global__ void __launch_bounds__(DEM_FUSED_THREADS, 1) dem_fused_kernel(DemArgs a, int npairs, int substeps) {
  const int slots = npairs + 6 * a.P;
  for (int s = 0; s < substeps; ++s) {
    for (int k = threadIdx.x; k < slots; k += blockDim.x) {
      if (k < npairs) {
        int i = 0, rem = k;
        while (rem >= a.P - 1 - i) { rem -= a.P - 1 - i; ++i; }
        pair_slot(a, i, i + 1 + rem);
      } else {
        const int w = k - npairs;
        wall_slot(a, w / 6, w % 6);
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < a.P; p += blockDim.x) integrate_particle(a, p);
    __syncthreads();
  }
}

__device__ void integrate_particle(const DemArgs& a, int p) {
  const int P = a.P;
  double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
  // slots not in contact hold no force: adding their zeros would change no bit, so they are skipped
  for (int j = 0; j < P; ++j) {
    if (j < p) {
      const size_t pr = (size_t)j * P + p;
      if (a.act[pr])
        for (int e = 0; e < 3; ++e) { F[e] = F[e] - a.pF[3 * pr + e]; T[e] = T[e] + a.pTj[3 * pr + e]; }
    } else if (j > p) {
      const size_t pr = (size_t)p * P + j;
      if (a.act[pr])
        for (int e = 0; e < 3; ++e) { F[e] = F[e] + a.pF[3 * pr + e]; T[e] = T[e] + a.pTi[3 * pr + e]; }
    }
  }
  for (int f = 0; f < 6; ++f)
    if (a.actw[6 * (size_t)p + f])
      for (int e = 0; e < 3; ++e) {
        F[e] = F[e] + a.wF[3 * (6 * (size_t)p + f) + e];
        T[e] = T[e] + a.wT[3 * (6 * (size_t)p + f) + e];
      }
  const double m = a.mass[p];
  for (int e = 0; e < 3; ++e) {
    if (a.Fe) { F[e] = F[e] + a.Fe[6 * p + e]; T[e] = T[e] + a.Fe[6 * p + 3 + e]; }
    F[e] = F[e] + m * a.g[e];
  }
  double* st = a.st + 13 * p;
  const double dt = a.dt;
  for (int e = 0; e < 3; ++e) {   // translation: symplectic Euler
    st[7 + e] = st[7 + e] + dt * (F[e] / m);
    st[e] = st[e] + dt * st[7 + e];
  }
  double R[3][3];   // rotation: I_w = R I_b R^T, w += dt I_w^-1 (T - w x I_w w)
  quat_matrix(st + 3, R);
  const double* I6 = a.Ib + 6 * p;
  const double Ib[3][3] = {{I6[0], I6[3], I6[4]}, {I6[3], I6[1], I6[5]}, {I6[4], I6[5], I6[2]}};
  double RI[3][3], Iw[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) RI[r][c] = R[r][0] * Ib[0][c] + R[r][1] * Ib[1][c] + R[r][2] * Ib[2][c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Iw[r][c] = RI[r][0] * R[c][0] + RI[r][1] * R[c][1] + RI[r][2] * R[c][2];
  double* w = st + 10;
  const double Lw[3] = {Iw[0][0] * w[0] + Iw[0][1] * w[1] + Iw[0][2] * w[2],
                        Iw[1][0] * w[0] + Iw[1][1] * w[1] + Iw[1][2] * w[2],
                        Iw[2][0] * w[0] + Iw[2][1] * w[1] + Iw[2][2] * w[2]};
  double gyro[3], dw[3];
  cross3(w, Lw, gyro);
  const double rhs[3] = {T[0] - gyro[0], T[1] - gyro[1], T[2] - gyro[2]};
  if (solve3(Iw, rhs, dw))
    for (int e = 0; e < 3; ++e) w[e] = w[e] + dt * dw[e];
  double* q = st + 3;   // orientation: q += dt/2 (0, w) q, normalised
  const double qw = q[0], qv[3] = {q[1], q[2], q[3]};
  double wxq[3];
  cross3(w, qv, wxq);
  const double h = 0.5 * dt;
  const double nq[4] = {qw - h * (w[0] * qv[0] + w[1] * qv[1] + w[2] * qv[2]),
                        qv[0] + h * (qw * w[0] + wxq[0]),
                        qv[1] + h * (qw * w[1] + wxq[1]),
                        qv[2] + h * (qw * w[2] + wxq[2])};
  const double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
  for (int e = 0; e < 4; ++e) q[e] = nq[e] / nn;
  a.posf[p] = make_float4((float)st[0], (float)st[1], (float)st[2], a.desc[p].rb);
}

// zoom s_p = 1 - R_s,p / R_c,p with R_c,p = max_i (|c_i| + sqrt(k_i)) over the body frame
__global__ void dem_init_kernel(DemArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  double r = 0.0;
  for (int i = a.desc[p].c0; i < a.desc[p].c1; ++i) {
    const float4 cb = a.cbody[i];
    const double x = (double)cb.x, y = (double)cb.y, z = (double)cb.z;
    const double e = sqrt(x * x + y * y + z * z) + sqrt((double)cb.w);
    if (e > r) r = e;
  }
  a.zoom[p] = 1.0 - a.Rs[p] / r;
  const double* st = a.st + 13 * p;
  a.posf[p] = make_float4((float)st[0], (float)st[1], (float)st[2], a.desc[p].rb);
}

// Mass properties from the metaball: body-frame sample points (i + 1/2) h, h = 1/4, out to the
// bound radius (N points per half-axis), inside when the binary32 sum reaches 1; integer sums in
// units of h/2 per particle: count, coordinates (3), products (xx yy zz xy xz yz). One block per
// particle; the sums are exact, so their order does not matter.
__global__ void dem_mass_sums_kernel(DemArgs a, unsigned long long* sums) {
  const int p = blockIdx.x;
  const ParticleDesc& d = a.desc[p];
  const int N = (int)ceil((double)d.rb / 0.25) + 1;
  const int side = 2 * N;
  const long long total = (long long)side * side * side;
  long long v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long m = threadIdx.x; m < total; m += blockDim.x) {
    const int i = (int)(m % side) - N, j = (int)((m / side) % side) - N, k = (int)(m / ((long long)side * side)) - N;
    const int ca = 2 * i + 1, cb = 2 * j + 1, cc = 2 * k + 1;
    const float x = (float)ca * 0.125f, y = (float)cb * 0.125f, z = (float)cc * 0.125f;
    float f = 0.0f;
    for (int q = d.c0; q < d.c1; ++q) {
      const float4 c = a.cbody[q];
      const float dx = x - c.x, dy = y - c.y, dz = z - c.z;
      const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
      float r2 = xx + yy;
      r2 = r2 + zz;
      f = f + c.w / r2;
    }
    if (f >= 1.0f) {
      v[0] += 1; v[1] += ca; v[2] += cb; v[3] += cc;
      v[4] += (long long)ca * ca; v[5] += (long long)cb * cb; v[6] += (long long)cc * cc;
      v[7] += (long long)ca * cb; v[8] += (long long)ca * cc; v[9] += (long long)cb * cc;
    }
  }
  for (int e = 0; e < 10; ++e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
    if ((threadIdx.x & 31) == 0 && v[e]) atomicAdd(&sums[10 * p + e], (unsigned long long)v[e]);
  }
}

// Per particle: mass, centre of mass and inertia about it (the oracle's formulas and order);
// moves the body frame to the centre of mass (control points c_i - c_m in binary32, state
// origin + c_m)
__global__ void dem_mass_finish_kernel(DemArgs a, const unsigned long long* sums, const double* density,
                                       double* mass, double* Ib, double* props, float4* cbody) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  long long S[10];
  for (int e = 0; e < 10; ++e) S[e] = (long long)sums[10 * p + e];
  const double dn = (double)S[0];
  const double rho = density[p];
  double* out = props + 10 * p;
  out[0] = rho * (dn * 0.015625);
  double cm[3];
  for (int e = 0; e < 3; ++e) { cm[e] = ((double)S[1 + e] * 0.125) / dn; out[1 + e] = cm[e]; }
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  double J[6];
  const double w = rho * 0.015625;
  for (int m = 0; m < 6; ++m) J[m] = ((double)S[4 + m] * 0.015625 - (dn * cm[ia[m]]) * cm[ib[m]]) * w;
  out[4] = J[1] + J[2];
  out[5] = J[0] + J[2];
  out[6] = J[0] + J[1];
  out[7] = -J[3];
  out[8] = -J[4];
  out[9] = -J[5];
  mass[p] = out[0];
  for (int m = 0; m < 6; ++m) Ib[6 * p + m] = out[4 + m];
  for (int q = a.desc[p].c0; q < a.desc[p].c1; ++q) {
    float4 c = cbody[q];
    c.x = (float)((double)c.x - cm[0]);
    c.y = (float)((double)c.y - cm[1]);
    c.z = (float)((double)c.z - cm[2]);
    cbody[q] = c;
  }
  for (int e = 0; e < 3; ++e) a.st[13 * p + e] = a.st[13 * p + e] + cm[e];
}

}  // namespace

void launch_dem_mass(const DemArgs& a, unsigned long long* sums, const double* density, double* mass, double* Ib,
                     double* props, float4* cbody, cudaStream_t st) {
  if (a.P <= 0) return;
  dem_mass_sums_kernel<<<(unsigned)a.P, 256, 0, st>>>(a, sums);
  dem_mass_finish_kernel<<<(unsigned)((a.P + 127) / 128), 128, 0, st>>>(a, sums, density, mass, Ib, props, cbody);
}

void launch_dem_init(const DemArgs& a, cudaStream_t st) {
  if (a.P > 0) dem_init_kernel<<<(unsigned)((a.P + 127) / 128), 128, 0, st>>>(a);
}

int launch_dem(const DemArgs& a, int substeps, cudaStream_t st) {
  if (a.P <= 0) return 0;
  const int npairs = a.P * (a.P - 1) / 2;
  if (a.P <= DEM_FUSED_MAX_P) {   // one block takes every step
    dem_fused_kernel<<<1, DEM_FUSED_THREADS, 0, st>>>(a, npairs, substeps);
    return 1;
  }
  const int slots = npairs + 6 * a.P;
  const unsigned cblocks = (unsigned)((slots + 63) / 64), iblocks = (unsigned)((a.P + 127) / 128);
  for (int s = 0; s < substeps; ++s) {
    dem_contacts_kernel<<<cblocks, 64, 0, st>>>(a, npairs);
    dem_integrate_kernel<<<iblocks, 128, 0, st>>>(a);
  }
  return 2 * substeps;
}

}  // namespace rwmi
