/*
 * rwmi_oracle.c -- plain, slow FP64 CPU reference ("the oracle") for one timestep of the
 * RW-MI-DELBM fluid-solute update (arXiv 2308.05007).
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite (with its mutation check), the package smoke check
 * and the benchmark's CPU baseline and reference legs are the only users of this library; the
 * product path never loads it. It shares no code, header, table or helper with the CUDA
 * library: the lattice tables, the counter-based generator, the metaball function and every
 * step below are written out here on their own.
 *
 * One timestep t -> t+1, in the order the oracle runs it:
 *   1. rigid particle poses at t and t+1: prescribed trajectories, or the free DEM of
 *      Eqs. 4-11 (sphero-metaball contacts, gravity, the fluid's force and torque);
 *   2. solid fraction per cell from the metaball function of Eq. 3 (4x4x4 sub-samples), or
 *      the solid/fluid node classes of the interpolated bounce-back;
 *   3. lattice Boltzmann pull-stream and collide, Eqs. 12-15 (D3Q19 as in Section 2.3, or
 *      D3Q15), with Guo body forcing and either partially-saturated-cell solid coupling or
 *      the paper's interpolated bounce-back, momentum exchange and refilling (Eqs. 23-27);
 *   4. random-walk advance of every solute walker, Eq. 2, with the four walker/particle
 *      relations of Section 2.4.2: free motion (I, III), Dirichlet refill (II), and the
 *      no-flux rule (IV) by Algorithm 1 (bisection) and Algorithm 2 (specular reflection);
 *   5. on request: concentration binning (Eq. 16), walker moments, mass/momentum, forces.
 *
 * Precision: FP64 throughout, except the two places where floating point decides an integer
 * that the GPU must reproduce exactly -- the sub-sample inside test of the solid fraction and
 * the accept/reject test of walker seeding. Those evaluate Eq. 3 in IEEE binary32 with a fixed
 * operation order (no contraction; build with -ffp-contract=off), which is the kernel's
 * precision. Readings of passages the paper leaves open are marked "Reading" below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------------
 * Counter-based generator: Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11). The paper only asks for a Gaussian
 * vector of zero mean and unit variance in Eq. 2; a counter-based generator keyed by
 * (walker id, step) makes every walker's noise independent of execution order.
 * ------------------------------------------------------------------------------------------ */
static void philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    for (int round = 0; round < 10; ++round) {
        /* S-box: two 32x32 -> 64-bit products, hi halves mixed with the other words and key */
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        /* key schedule: Weyl sequence with the golden-ratio and sqrt(3)-1 constants */
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* U = ((r >> 8) + 1/2) 2^-24: 24-bit uniform strictly inside (0, 1), exact in FP32 and FP64 */
static double u24(uint32_t r) { return ((double)(r >> 8) + 0.5) * 5.9604644775390625e-08; }

/* Box-Muller transform of two uniforms into two independent standard normals */
static void box_muller(double ua, double ub, double* za, double* zb)
{
    double rad = sqrt(-2.0 * log(ua));
    double ang = 2.0 * M_PI * ub;
    *za = rad * cos(ang);
    if (zb) *zb = rad * sin(ang);
}

/* ------------------------------------------------------------------------------------------
 * Lattice velocity sets. Section 2.3 names D3Q19 (the sums of Eqs. 14-15 run over 19
 * directions); D3Q15 is offered as well. Weights and c_s^2 = 1/3 are the standard ones of
 * Qian, d'Humieres and Lallemand (1992). Directions come in opposite pairs (2m-1, 2m).
 * ------------------------------------------------------------------------------------------ */
static const int E15[15][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
static const int E19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double lattice_weight(int q, int i)
{
    if (q == 15) return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}
static const int* lattice_e(int q, int i) { return q == 15 ? E15[i] : E19[i]; }
static int opposite(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

/* ------------------------------------------------------------------------------------------
 * State
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int n[3];
    long long ncell;
    int q;
    double tau, D;
    uint32_t key0, key1;
    int wall[3];             /* no-slip walls on the two faces normal to this axis */
    double F0[3], Fperiod;   /* body force density F(t) = F0 sin(2 pi t / Fperiod), or F0 */
    double rho0, u_init[3];

    /* metaball particles (Eq. 3), rigid, prescribed motion */
    int P, Nc;
    int* coff;               /* [P+1] */
    double* cbody;           /* [3 Nc] body-frame control points */
    double* kc;              /* [Nc] */
    float* kc32;             /* [Nc] the same weights as given (binary32) */
    double *org, *amp, *per, *pha, *omg;   /* [3P] [3P] [P] [P] [3P] */
    double* Rb;              /* [P] bound: f_p < 1 farther than Rb from the origin */

    /* fluid */
    double *f, *fn;          /* [q ncell], direction-major; f holds post-collision of t-1 */
    double *u, *rho;         /* [3 ncell], [ncell] of the last LBM step */
    int *cnt, *own;          /* solid sub-sample count 0..64 and owner per cell, time t */
    long long solid_time;
    double mass, mom[3];     /* sums over cells of rho and sum_i f_i e_i, last LBM step */
    double *Fp, *Tp;         /* [3P] hydrodynamic force and torque, last LBM step */

    /* walkers */
    long long nw;
    double *x, *x0;          /* [3 nw] unwrapped positions and start positions */

    long long t;
    long long cnt_type[4], bisect_fail, refill_fail, wall_fail, seed_fail;

    int coupling;            /* 0: partially saturated cells; 1: IBB + momentum exchange + refilling */

    /* free DEM (Eqs. 4-11), active once orc_set_dem is called */
    int dem, dem_nsub, dem_hydro;
    double dem_kn, dem_etan, dem_kt, dem_etat, dem_mus, dem_g[3];
    double* dst;             /* [13 P] origin (unwrapped), quaternion (w, x, y, z), velocity, spin */
    double *dmass, *dIb, *dRs, *dzoom;   /* [P], [6 P] body inertia (xx yy zz xy xz yz), [P], [P] */
    double* dcm;             /* [10 P] mass properties (orc_dem_mass) */
    int* dem_nodes;          /* IBB node classes of the last LBM step (free DEM) */
    long long dem_nodes_t;
    double *dxi, *dxm;       /* pairs (i < j) at i P + j: tangential spring, Newton point [3 each] */
    unsigned char* dact;     /* pair in contact at the last DEM step */
    double *dxiw, *dxmw;     /* walls: particle p, face f (2 axis + side) at 6 p + f */
    unsigned char* dactw;
} orc_t;

static long long cell_index(const orc_t* o, long long i, long long j, long long k)
{
    return (k * o->n[1] + j) * o->n[0] + i;
}

static long long wrapll(long long a, long long n) { a %= n; return a < 0 ? a + n : a; }

/* ------------------------------------------------------------------------------------------
 * Prescribed particle motion (stand-in for Eq. 4; Eq. 37 drives the oscillator case with a
 * sinusoid). Origin o(t) = o0 + A sin(2 pi t / T + phi), velocity its time derivative,
 * constant spin omega: the body frame turns by |omega| t about omega/|omega| (Rodrigues).
 * ------------------------------------------------------------------------------------------ */
static void particle_pose(const orc_t* o, long long t, int p, double org[3], double vel[3],
                          double R[3][3])
{
    double s = 0.0, cdt = 0.0;
    if (o->per[p] > 0.0) {
        double th = 2.0 * M_PI * (double)t / o->per[p] + o->pha[p];
        s = sin(th);
        cdt = cos(th) * 2.0 * M_PI / o->per[p];
    }
    for (int a = 0; a < 3; ++a) {
        org[a] = o->org[3 * p + a] + o->amp[3 * p + a] * s;
        vel[a] = o->amp[3 * p + a] * cdt;
    }
    double w[3] = {o->omg[3 * p], o->omg[3 * p + 1], o->omg[3 * p + 2]};
    double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[a][b] = (a == b) ? 1.0 : 0.0;
    if (wn > 0.0) {
        double ax[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
        double ang = wn * (double)t, ca = cos(ang), sa = sin(ang);
        /* R = cos I + sin [n]x + (1 - cos) n n^T */
        double K[3][3] = {{0, -ax[2], ax[1]}, {ax[2], 0, -ax[0]}, {-ax[1], ax[0], 0}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                R[a][b] = (a == b ? ca : 0.0) + sa * K[a][b] + (1.0 - ca) * ax[a] * ax[b];
    }
}

/* Origin wrapped into the box on periodic axes */
static void wrap_point(const orc_t* o, double x[3])
{
    for (int a = 0; a < 3; ++a)
        if (!o->wall[a]) x[a] -= (double)o->n[a] * floor(x[a] / (double)o->n[a]);
}

/* World positions of all control points at time t (wrapped on periodic axes), plus each
 * particle's wrapped origin and velocity, in FP64 and rounded to binary32. */
typedef struct {
    double* c;    /* [3 Nc] */
    float* c32;   /* [3 Nc] */
    double* o;    /* [3 P] wrapped origin */
    double* v;    /* [3 P] */
    double* w;    /* [3 P] spin */
} frame_t;

static void frame_alloc(const orc_t* o, frame_t* fr)
{
    fr->c = (double*)calloc(3 * (size_t)o->Nc + 3, sizeof(double));
    fr->c32 = (float*)calloc(3 * (size_t)o->Nc + 3, sizeof(float));
    fr->o = (double*)calloc(3 * (size_t)o->P + 3, sizeof(double));
    fr->v = (double*)calloc(3 * (size_t)o->P + 3, sizeof(double));
    fr->w = (double*)calloc(3 * (size_t)o->P + 3, sizeof(double));
}
static void frame_free(frame_t* fr) { free(fr->c); free(fr->c32); free(fr->o); free(fr->v); free(fr->w); }

static void dem_pose(const orc_t* o, int p, double org[3], double vel[3], double R[3][3]);

/* With the free DEM only the current state exists: every t reads it (the stepping order below
 * asks for the frame of the state's own time). */
static void frame_at(const orc_t* o, long long t, frame_t* fr)
{
    for (int p = 0; p < o->P; ++p) {
        double org[3], vel[3], R[3][3];
        if (o->dem) dem_pose(o, p, org, vel, R);
        else particle_pose(o, t, p, org, vel, R);
        for (int i = o->coff[p]; i < o->coff[p + 1]; ++i) {
            double cw[3];
            for (int a = 0; a < 3; ++a)
                cw[a] = org[a] + R[a][0] * o->cbody[3 * i] + R[a][1] * o->cbody[3 * i + 1]
                        + R[a][2] * o->cbody[3 * i + 2];
            wrap_point(o, cw);
            for (int a = 0; a < 3; ++a) { fr->c[3 * i + a] = cw[a]; fr->c32[3 * i + a] = (float)cw[a]; }
        }
        wrap_point(o, org);
        for (int a = 0; a < 3; ++a) {
            fr->o[3 * p + a] = org[a];
            fr->v[3 * p + a] = vel[a];
            fr->w[3 * p + a] = o->dem ? o->dst[13 * p + 10 + a] : o->omg[3 * p + a];
        }
    }
}

/* Minimum-image displacement on periodic axes (Reading: a metaball near a periodic face acts
 * through it, as the fluid and walkers do). Both arguments lie in [0, n). */
static double min_image(const orc_t* o, int a, double d)
{
    if (!o->wall[a]) {
        double n = (double)o->n[a];
        if (d > 0.5 * n) d -= n;
        else if (d < -0.5 * n) d += n;
    }
    return d;
}

/* Eq. 3, f(x) = sum_i k_i / |x - x_i|^2, and its gradient, Eq. 17,
 * grad f = sum_i -2 k_i (x - x_i) / |x - x_i|^4, for particle p; x wrapped into the box. */
static double metaball64(const orc_t* o, const frame_t* fr, int p, const double x[3], double g[3])
{
    double f = 0.0;
    if (g) g[0] = g[1] = g[2] = 0.0;
    for (int i = o->coff[p]; i < o->coff[p + 1]; ++i) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = min_image(o, a, x[a] - fr->c[3 * i + a]);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        f += o->kc[i] / r2;
        if (g) {
            double s = -2.0 * o->kc[i] / (r2 * r2);
            for (int a = 0; a < 3; ++a) g[a] += s * d[a];
        }
    }
    return f;
}

/* Eq. 3 in binary32 with a fixed operation order: the inside test that decides sub-sample
 * counts and seeding accept/reject. d = x - c, one minimum-image correction by +-n, then
 * r2 = (dx*dx + dy*dy) + dz*dz and f = ((k_0/r2_0) + k_1/r2_1) + ... */
static float metaball32(const orc_t* o, const frame_t* fr, int p, const float x[3])
{
    float f = 0.0f;
    for (int i = o->coff[p]; i < o->coff[p + 1]; ++i) {
        float d[3];
        for (int a = 0; a < 3; ++a) {
            float da = x[a] - fr->c32[3 * i + a];
            if (!o->wall[a]) {
                float n = (float)o->n[a];
                float h = 0.5f * n;
                if (da > h) da = da - n;
                else if (da < -h) da = da + n;
            }
            d[a] = da;
        }
        float xx = d[0] * d[0];
        float yy = d[1] * d[1];
        float zz = d[2] * d[2];
        float r2 = xx + yy;
        r2 = r2 + zz;
        float term = o->kc32[i] / r2;
        f = f + term;
    }
    return f;
}

/* Distance from x (wrapped) to particle p's wrapped origin, minimum image */
static double origin_distance(const orc_t* o, const frame_t* fr, int p, const double x[3])
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double d = min_image(o, a, x[a] - fr->o[3 * p + a]);
        s += d * d;
    }
    return sqrt(s);
}

/* Bound on a particle's extent. With r = |x - o| and |x - x_i| >= r - |c_i| for every
 * control point, f(x) <= sum_i k_i / (r - |c_i|)^2 once r > max |c_i|; the right side falls
 * monotonically, so beyond its unit crossing Rb every point has f < 1 (Eq. 3 is exact here,
 * the bound only lets a cell or walker skip a particle it cannot touch). */
static double bound_radius(const orc_t* o, int p)
{
    double cmax = 0.0, ksum = 0.0;
    for (int i = o->coff[p]; i < o->coff[p + 1]; ++i) {
        double c = sqrt(o->cbody[3 * i] * o->cbody[3 * i] + o->cbody[3 * i + 1] * o->cbody[3 * i + 1]
                        + o->cbody[3 * i + 2] * o->cbody[3 * i + 2]);
        if (c > cmax) cmax = c;
        ksum += o->kc[i];
    }
    double lo = cmax, hi = cmax + sqrt(ksum) + 1e-9;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), s = 0.0;
        for (int i = o->coff[p]; i < o->coff[p + 1]; ++i) {
            double c = sqrt(o->cbody[3 * i] * o->cbody[3 * i] + o->cbody[3 * i + 1] * o->cbody[3 * i + 1]
                            + o->cbody[3 * i + 2] * o->cbody[3 * i + 2]);
            s += o->kc[i] / ((mid - c) * (mid - c));
        }
        if (s > 1.0) lo = mid; else hi = mid;
    }
    return hi;
}

/* Lowest-index particle whose metaball reaches 1 at x (FP64); -1 if x is in the fluid */
static int inside_any64(const orc_t* o, const frame_t* fr, const double xin[3])
{
    double x[3] = {xin[0], xin[1], xin[2]};
    wrap_point(o, x);
    for (int p = 0; p < o->P; ++p) {
        if (origin_distance(o, fr, p, x) > o->Rb[p] + 1e-6) continue;
        if (metaball64(o, fr, p, x, NULL) >= 1.0) return p;
    }
    return -1;
}

/* The same test in binary32 (seeding accept/reject) */
static int inside_any32(const orc_t* o, const frame_t* fr, const float x[3])
{
    double xd[3] = {x[0], x[1], x[2]};
    for (int p = 0; p < o->P; ++p) {
        if (origin_distance(o, fr, p, xd) > o->Rb[p] + 0.5) continue;
        if (metaball32(o, fr, p, x) >= 1.0f) return p;
    }
    return -1;
}

/* ------------------------------------------------------------------------------------------
 * Solid fraction per cell. The partially-saturated-cells method is named in Section 1; the
 * paper gives no formula for the fraction. Reading: node at the cell centre, cell
 * [i, i+1) x [j, j+1) x [k, k+1); 4x4x4 sub-samples at i + (a + 1/2)/4 etc.; a sub-sample is
 * solid when some particle's Eq. 3 value is >= 1 there; the count n (0..64) gives
 * epsilon = n / 64. Owner: the particle holding the most sub-samples, lowest index on ties.
 * Every sub-sample of every cell is tested; a particle is skipped for a cell only when the
 * cell lies wholly beyond its bound radius, where Eq. 3 stays below 1.
 * ------------------------------------------------------------------------------------------ */
/* Solid fraction of one cell (Reading R3): sub-sample count and owner of cell (i, j, k) against
 * the poses in fr. cand and npart are scratch arrays of P + 1 ints. */
static void raster_cell(const orc_t* o, const frame_t* fr, long long i, long long j, long long k,
                        int* cand, int* npart, int* cnt_out, int* own_out)
{
    double xc[3] = {i + 0.5, j + 0.5, k + 0.5};
    int nc = 0;
    for (int p = 0; p < o->P; ++p)
        if (origin_distance(o, fr, p, xc) <= o->Rb[p] + 1.0) { cand[nc++] = p; npart[p] = 0; }
    int count = 0;
    if (nc > 0) {
        for (int cz = 0; cz < 4; ++cz)
            for (int cy = 0; cy < 4; ++cy)
                for (int cx = 0; cx < 4; ++cx) {
                    float xs[3] = {(float)i + (0.125f + 0.25f * (float)cx),
                                   (float)j + (0.125f + 0.25f * (float)cy),
                                   (float)k + (0.125f + 0.25f * (float)cz)};
                    int solid = 0;
                    for (int m = 0; m < nc; ++m)
                        if (metaball32(o, fr, cand[m], xs) >= 1.0f) { npart[cand[m]]++; solid = 1; }
                    count += solid;
                }
    }
    int owner = -1, best = 0;
    for (int m = 0; m < nc; ++m)
        if (npart[cand[m]] > best) { best = npart[cand[m]]; owner = cand[m]; }
    *cnt_out = count;
    *own_out = count > 0 ? owner : -1;
}

static void rasterize(orc_t* o, long long t)
{
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    int* cand = (int*)malloc(sizeof(int) * (size_t)(o->P + 1));
    int* npart = (int*)calloc((size_t)o->P + 1, sizeof(int));
    for (long long k = 0; k < o->n[2]; ++k)
        for (long long j = 0; j < o->n[1]; ++j)
            for (long long i = 0; i < o->n[0]; ++i) {
                long long c = cell_index(o, i, j, k);
                raster_cell(o, &fr, i, j, k, cand, npart, &o->cnt[c], &o->own[c]);
            }
    free(cand);
    free(npart);
    frame_free(&fr);
    o->solid_time = t;
}

/* Body force density at step t (Reading: a force density F, as rho0 g with rho0 = 1) */
static void body_force(const orc_t* o, long long t, double F[3])
{
    double s = 1.0;
    if (o->Fperiod > 0.0) s = sin(2.0 * M_PI * (double)t / o->Fperiod);
    for (int a = 0; a < 3; ++a) F[a] = o->F0[a] * s;
}

/* Eq. 13: second-order equilibrium with c_s^2 = 1/3 */
static double feq(int q, int i, double rho, const double u[3])
{
    const int* e = lattice_e(q, i);
    double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return lattice_weight(q, i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* Post-collision populations of one cell at step t from the pulled populations fi.
 *  - Eqs. 14-15 moments; velocity with half the body force (Guo, Zheng and Shi 2002):
 *    u = (sum_i f_i e_i + F/2) / rho.
 *  - Eq. 12 BGK relaxation towards Eq. 13, weighted by the fluid share (1 - B).
 *  - Partially saturated cells (Noble and Torczynski 1998): B = eps (tau - 1/2) /
 *    ((1 - eps) + (tau - 1/2)), solid term Omega_i = f_opp(i) - feq_opp(i)(rho, u)
 *    - f_i + feq_i(rho, u_s), with u_s = v_p + omega_p x (x - o_p) of the owner particle.
 *  - Guo source S_i = (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F, weighted by
 *    (1 - B).
 * Returns the momentum the solid term puts into the fluid, B sum_i Omega_i e_i, in dp. */
static void collide_cell(const orc_t* o, const frame_t* fr, long long t, long long i, long long j,
                         long long k, int count, int owner, const double fi[19], const double F[3],
                         double fout[19], double u[3], double* rho_out, double dp[3])
{
    int q = o->q;
    double tau = o->tau;
    double rho = 0.0, jm[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < q; ++m) {
        const int* e = lattice_e(q, m);
        rho += fi[m];
        for (int a = 0; a < 3; ++a) jm[a] += fi[m] * e[a];
    }
    for (int a = 0; a < 3; ++a) u[a] = (jm[a] + 0.5 * F[a]) / rho;
    *rho_out = rho;
    double eps = count / 64.0;
    double B = eps * (tau - 0.5) / ((1.0 - eps) + (tau - 0.5));
    double us[3] = {0.0, 0.0, 0.0};
    if (B > 0.0 && owner >= 0) {
        double r[3];
        double xn[3] = {i + 0.5, j + 0.5, k + 0.5};
        for (int a = 0; a < 3; ++a) r[a] = min_image(o, a, xn[a] - fr->o[3 * owner + a]);
        const double* v = fr->v + 3 * owner;
        const double* w = fr->w + 3 * owner;
        us[0] = v[0] + w[1] * r[2] - w[2] * r[1];
        us[1] = v[1] + w[2] * r[0] - w[0] * r[2];
        us[2] = v[2] + w[0] * r[1] - w[1] * r[0];
    }
    dp[0] = dp[1] = dp[2] = 0.0;
    double guo = 1.0 - 0.5 / tau;
    for (int m = 0; m < q; ++m) {
        const int* e = lattice_e(q, m);
        double w = lattice_weight(q, m);
        double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        double S = 0.0;
        for (int a = 0; a < 3; ++a) S += (3.0 * (e[a] - u[a]) + 9.0 * eu * e[a]) * F[a];
        S *= guo * w;
        double fe = feq(q, m, rho, u);
        double om = 0.0;
        if (B > 0.0) {
            int mo = opposite(m);
            om = fi[mo] - feq(q, mo, rho, u) - fi[m] + feq(q, m, rho, us);
            for (int a = 0; a < 3; ++a) dp[a] += B * om * e[a];
        }
        fout[m] = fi[m] - (1.0 - B) * (fi[m] - fe) / tau + B * om + (1.0 - B) * S;
    }
    (void)t;
}

/* Pull streaming, Eq. 12 left side: f_i(x, t) = f+_i(x - e_i, t - 1) with periodic wrap;
 * where x - e_i lies beyond a wall the half-way bounce-back f_i(x, t) = f+_opp(i)(x, t - 1)
 * applies (the wall sits on the cell face, at rest). */
static void pull_cell(const orc_t* o, long long i, long long j, long long k, double fi[19])
{
    long long c = cell_index(o, i, j, k);
    for (int m = 0; m < o->q; ++m) {
        const int* e = lattice_e(o->q, m);
        long long s[3] = {i - e[0], j - e[1], k - e[2]};
        int blocked = 0;
        for (int a = 0; a < 3; ++a) {
            if (o->wall[a]) {
                if (s[a] < 0 || s[a] >= o->n[a]) blocked = 1;
            } else {
                s[a] = wrapll(s[a], o->n[a]);
            }
        }
        if (blocked) fi[m] = o->f[(size_t)opposite(m) * o->ncell + c];
        else fi[m] = o->f[(size_t)m * o->ncell + cell_index(o, s[0], s[1], s[2])];
    }
}

static void ibb_step(orc_t* o, long long t);

static void lbm_step(orc_t* o, long long t)
{
    if (o->coupling == 1) { ibb_step(o, t); return; }
    if (o->solid_time != t) rasterize(o, t);
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    double F[3];
    body_force(o, t, F);
    o->mass = 0.0;
    o->mom[0] = o->mom[1] = o->mom[2] = 0.0;
    for (int m = 0; m < 3 * o->P; ++m) { o->Fp[m] = 0.0; o->Tp[m] = 0.0; }
    for (long long k = 0; k < o->n[2]; ++k)
        for (long long j = 0; j < o->n[1]; ++j)
            for (long long i = 0; i < o->n[0]; ++i) {
                long long c = cell_index(o, i, j, k);
                double fi[19], fo[19], u[3], rho, dp[3];
                pull_cell(o, i, j, k, fi);
                collide_cell(o, &fr, t, i, j, k, o->cnt[c], o->own[c], fi, F, fo, u, &rho, dp);
                for (int m = 0; m < o->q; ++m) o->fn[(size_t)m * o->ncell + c] = fo[m];
                for (int a = 0; a < 3; ++a) o->u[3 * c + a] = u[a];
                o->rho[c] = rho;
                o->mass += rho;
                for (int m = 0; m < o->q; ++m) {
                    const int* e = lattice_e(o->q, m);
                    for (int a = 0; a < 3; ++a) o->mom[a] += fi[m] * e[a];
                }
                int p = o->own[c];
                if (o->cnt[c] > 0 && p >= 0) {
                    /* force on the particle: the opposite of what the solid term gives the
                     * fluid; torque about the particle origin (minimum image) */
                    double Fc[3] = {-dp[0], -dp[1], -dp[2]}, r[3];
                    double xn[3] = {i + 0.5, j + 0.5, k + 0.5};
                    for (int a = 0; a < 3; ++a) r[a] = min_image(o, a, xn[a] - fr.o[3 * p + a]);
                    for (int a = 0; a < 3; ++a) o->Fp[3 * p + a] += Fc[a];
                    o->Tp[3 * p + 0] += r[1] * Fc[2] - r[2] * Fc[1];
                    o->Tp[3 * p + 1] += r[2] * Fc[0] - r[0] * Fc[2];
                    o->Tp[3 * p + 2] += r[0] * Fc[1] - r[1] * Fc[0];
                }
            }
    double* tmp = o->f;
    o->f = o->fn;
    o->fn = tmp;
    frame_free(&fr);
}

/* ------------------------------------------------------------------------------------------
 * The paper's own particle-fluid coupling, Section 2.4.3, used instead of partially saturated
 * cells when coupling = 1: interpolated bounce-back on the moving particle surface (Eqs. 23-25),
 * Galilean-invariant momentum exchange for the force, local refilling (Eqs. 26-27).
 * Readings (the paper leaves these open):
 *  - A node (cell centre) is solid at time t when Eq. 3 of some particle reaches c0 = 1 there,
 *    decided in binary32 with the fixed operation order of metaball32; it belongs to the lowest
 *    such particle index.
 *  - q of Eq. 25: the fraction of the link from the fluid node x_f to the solid node at which
 *    Eq. 3 of the solid node's particle crosses 1: 24 bisection steps in binary32 (midpoint
 *    0.5 (lo + hi), link point x_f + mid e), q = the middle of the last bracket.
 *  - u_f, u_ff and rho_f are the velocity and density of the previous LBM update (rho_f as the
 *    sum of x_f's own post-collision populations, which carry the same mass); x_ff = x_f + e_i,
 *    one node further from the wall, and u_ff = u_f when x_ff is solid or beyond a wall.
 *  - The non-equilibrium part G^neq_i'(x_d) of Eq. 24 is taken at x_f:
 *    G+_i'(x_f, t) - G^eq_i'(rho_f, u_f).
 *  - Force on the particle per link (Galilean-invariant momentum exchange, Wen et al. 2014):
 *    (e_i' - u_w) G+_i'(x_f) - (e_i - u_w) G_i(x_f, t + 1); torque (x_w - o_p) x that force,
 *    with x_w = x_f + q e_i' the wall point and u_w the particle's rigid velocity there.
 *  - Refilling: a node solid at t - 1 and fluid at t has no populations of its own, so Eq. 26's
 *    G_i' does not exist and Eq. 27 applies: G^eq(rho0, u_new), u_new the covering
 *    particle's rigid velocity at the node at time t.
 *  - Solid nodes hold G^eq(rho0, u_s) at their particle's rigid velocity u_s and report u_s
 *    (the walkers interpolate it); the mass and momentum sums count fluid nodes only.
 * ------------------------------------------------------------------------------------------ */

/* Rigid velocity of particle p at x: v_p + omega_p x (x - o_p), minimum image */
static void rigid_velocity(const orc_t* o, const frame_t* fr, int p, const double x[3], double u[3])
{
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = min_image(o, a, x[a] - fr->o[3 * p + a]);
    const double* v = fr->v + 3 * p;
    const double* w = fr->w + 3 * p;
    u[0] = v[0] + w[1] * r[2] - w[2] * r[1];
    u[1] = v[1] + w[2] * r[0] - w[0] * r[2];
    u[2] = v[2] + w[0] * r[1] - w[1] * r[0];
}

/* Node classes at time t: node[c] = 1 + the lowest particle whose Eq. 3 reaches 1 at the cell
 * centre (binary32 decision), 0 for a fluid node. */
static void classify_nodes(const orc_t* o, long long t, int* node)
{
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    for (long long k = 0; k < o->n[2]; ++k)
        for (long long j = 0; j < o->n[1]; ++j)
            for (long long i = 0; i < o->n[0]; ++i) {
                long long c = cell_index(o, i, j, k);
                double xc[3] = {i + 0.5, j + 0.5, k + 0.5};
                float xs[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
                node[c] = 0;
                for (int p = 0; p < o->P; ++p)
                    if (origin_distance(o, &fr, p, xc) <= o->Rb[p] + 1.0 && metaball32(o, &fr, p, xs) >= 1.0f) {
                        node[c] = p + 1;
                        break;
                    }
            }
    frame_free(&fr);
}

/* q of Eq. 25 on the link from node (i, j, k) along e (towards particle p's solid node) */
static float ibb_q(const orc_t* o, const frame_t* fr, int p, long long i, long long j, long long k, const int* e)
{
    const float x0[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
    float lo = 0.0f, hi = 1.0f;
    for (int it = 0; it < 24; ++it) {
        float mid = 0.5f * (lo + hi);
        float xm[3];
        for (int a = 0; a < 3; ++a) {
            float step = mid * (float)e[a];
            xm[a] = x0[a] + step;
        }
        if (metaball32(o, fr, p, xm) >= 1.0f) hi = mid;
        else lo = mid;
    }
    return 0.5f * (lo + hi);
}

/* Eqs. 23-25 for one link: the population G_i(x_f, t + 1) entering x_f from the wall, i the
 * direction away from the wall and ip = opposite(i) the direction into it. */
static double ibb_link(int q, int i, int ip, double qf, double rho_f, const double uf[3], const double uff[3],
                       const double uw[3], double Gp)
{
    double us[3], uss[3], ud[3];
    for (int a = 0; a < 3; ++a) {
        if (qf <= 0.5) us[a] = 2.0 * qf * uf[a] + (1.0 - 2.0 * qf) * uff[a];
        else us[a] = (1.0 - qf) / qf * uf[a] + (2.0 * qf - 1.0) / qf * uw[a];
        uss[a] = (1.0 - qf) / (1.0 + qf) * uff[a] + 2.0 * qf / (1.0 + qf) * uw[a];
        ud[a] = us[a] / 3.0 + 2.0 * uss[a] / 3.0;
    }
    const int* e = lattice_e(q, i);
    double eu = e[0] * uw[0] + e[1] * uw[1] + e[2] * uw[2];
    double gneq = Gp - feq(q, ip, rho_f, uf);
    return feq(q, ip, rho_f, ud) + gneq + 6.0 * lattice_weight(q, ip) * rho_f * eu;
}

static void ibb_step(orc_t* o, long long t)
{
    const int q = o->q;
    const long long n = o->ncell;
    int* nprev = (int*)malloc(sizeof(int) * (size_t)n);
    int* ncur = (int*)malloc(sizeof(int) * (size_t)n);
    double* uprev = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(uprev, o->u, sizeof(double) * 3 * (size_t)n);
    classify_nodes(o, t, ncur);
    /* With the free DEM only the current particle state exists: the classes of t - 1 are those
     * this step stored at the previous time, and at the first step of a run the classes of t
     * (nothing is refilled then). */
    if (!o->dem) classify_nodes(o, t - 1, nprev);
    else if (o->dem_nodes_t == t - 1) memcpy(nprev, o->dem_nodes, sizeof(int) * (size_t)n);
    else memcpy(nprev, ncur, sizeof(int) * (size_t)n);
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    double F[3];
    body_force(o, t, F);
    /* refilling of nodes uncovered since t - 1, Eq. 27 */
    for (long long k = 0; k < o->n[2]; ++k)
        for (long long j = 0; j < o->n[1]; ++j)
            for (long long i = 0; i < o->n[0]; ++i) {
                long long c = cell_index(o, i, j, k);
                if (nprev[c] == 0 || ncur[c] != 0) continue;
                double xc[3] = {i + 0.5, j + 0.5, k + 0.5}, un[3];
                rigid_velocity(o, &fr, nprev[c] - 1, xc, un);
                for (int m = 0; m < q; ++m) o->f[(size_t)m * n + c] = feq(q, m, o->rho0, un);
            }
    o->mass = 0.0;
    o->mom[0] = o->mom[1] = o->mom[2] = 0.0;
    for (int m = 0; m < 3 * o->P; ++m) { o->Fp[m] = 0.0; o->Tp[m] = 0.0; }
    for (long long k = 0; k < o->n[2]; ++k)
        for (long long j = 0; j < o->n[1]; ++j)
            for (long long i = 0; i < o->n[0]; ++i) {
                long long c = cell_index(o, i, j, k);
                double xc[3] = {i + 0.5, j + 0.5, k + 0.5};
                if (ncur[c] != 0) {   /* solid node */
                    double us[3];
                    rigid_velocity(o, &fr, ncur[c] - 1, xc, us);
                    for (int m = 0; m < q; ++m) o->fn[(size_t)m * n + c] = feq(q, m, o->rho0, us);
                    for (int a = 0; a < 3; ++a) o->u[3 * c + a] = us[a];
                    o->rho[c] = o->rho0;
                    continue;
                }
                double fi[19], fo[19], u[3], rho, dp[3];
                pull_cell(o, i, j, k, fi);
                double rho_f = 0.0;
                for (int m = 0; m < q; ++m) rho_f += o->f[(size_t)m * n + c];
                const double* uf = uprev + 3 * c;
                long long ijk[3] = {i, j, k};
                for (int m = 0; m < q; ++m) {
                    const int* e = lattice_e(q, m);
                    long long s[3], ff[3];
                    int blocked = 0, ff_out = 0;
                    for (int a = 0; a < 3; ++a) {
                        s[a] = ijk[a] - e[a];
                        ff[a] = ijk[a] + e[a];
                        if (o->wall[a]) {
                            if (s[a] < 0 || s[a] >= o->n[a]) blocked = 1;
                            if (ff[a] < 0 || ff[a] >= o->n[a]) ff_out = 1;
                        } else {
                            s[a] = wrapll(s[a], o->n[a]);
                            ff[a] = wrapll(ff[a], o->n[a]);
                        }
                    }
                    if (blocked) continue;                       /* plane wall: bounce-back above */
                    long long cs = cell_index(o, s[0], s[1], s[2]);
                    if (ncur[cs] == 0) continue;                 /* fluid source: plain pull */
                    const int p = ncur[cs] - 1, ip = opposite(m);
                    const int* eip = lattice_e(q, ip);
                    const double qf = (double)ibb_q(o, &fr, p, i, j, k, eip);
                    double xw[3], uw[3];
                    for (int a = 0; a < 3; ++a) xw[a] = xc[a] + qf * eip[a];
                    rigid_velocity(o, &fr, p, xw, uw);
                    const double* uff = uf;
                    if (!ff_out) {
                        long long cf = cell_index(o, ff[0], ff[1], ff[2]);
                        if (ncur[cf] == 0) uff = uprev + 3 * cf;
                    }
                    const double Gp = o->f[(size_t)ip * n + c];
                    fi[m] = ibb_link(q, m, ip, qf, rho_f, uf, uff, uw, Gp);
                    double Fl[3], r[3];
                    for (int a = 0; a < 3; ++a) Fl[a] = (eip[a] - uw[a]) * Gp - (e[a] - uw[a]) * fi[m];
                    for (int a = 0; a < 3; ++a) r[a] = min_image(o, a, xw[a] - fr.o[3 * p + a]);
                    for (int a = 0; a < 3; ++a) o->Fp[3 * p + a] += Fl[a];
                    o->Tp[3 * p + 0] += r[1] * Fl[2] - r[2] * Fl[1];
                    o->Tp[3 * p + 1] += r[2] * Fl[0] - r[0] * Fl[2];
                    o->Tp[3 * p + 2] += r[0] * Fl[1] - r[1] * Fl[0];
                }
                collide_cell(o, &fr, t, i, j, k, 0, -1, fi, F, fo, u, &rho, dp);
                for (int m = 0; m < q; ++m) o->fn[(size_t)m * n + c] = fo[m];
                for (int a = 0; a < 3; ++a) o->u[3 * c + a] = u[a];
                o->rho[c] = rho;
                o->mass += rho;
                for (int m = 0; m < q; ++m) {
                    const int* e = lattice_e(q, m);
                    for (int a = 0; a < 3; ++a) o->mom[a] += fi[m] * e[a];
                }
            }
    double* tmp = o->f;
    o->f = o->fn;
    o->fn = tmp;
    frame_free(&fr);
    free(nprev);
    if (o->dem) {   /* the classes of t, for the next step */
        if (!o->dem_nodes) o->dem_nodes = (int*)malloc(sizeof(int) * (size_t)n);
        memcpy(o->dem_nodes, ncur, sizeof(int) * (size_t)n);
        o->dem_nodes_t = t;
    }
    free(ncur);
    free(uprev);
}

/* ------------------------------------------------------------------------------------------
 * Random-walk method, Section 2.4
 * ------------------------------------------------------------------------------------------ */

/* Section 2.4.1: the walker takes the fluid velocity by linear interpolation from the LBM
 * grid. Reading: trilinear over the eight nodes (cell centres) around x, periodic wrap on
 * periodic axes; on a walled axis the wall plane carries u = 0 and the half cell between the
 * wall and the first node interpolates linearly to it. */
static void axis_stencil(const orc_t* o, int a, double xa, long long idx[2], double wt[2])
{
    long long n = o->n[a];
    if (!o->wall[a]) {
        double s = xa - 0.5;
        double fl = floor(s);
        double w = s - fl;
        long long i0 = (long long)fl;
        idx[0] = wrapll(i0, n);
        idx[1] = wrapll(i0 + 1, n);
        wt[0] = 1.0 - w;
        wt[1] = w;
        return;
    }
    if (xa < 0.0) xa = 0.0;
    if (xa > (double)n) xa = (double)n;
    if (xa < 0.5) {                       /* wall at 0 (value 0) .. node 0 at 0.5 */
        idx[0] = -1; idx[1] = 0;
        wt[1] = xa / 0.5; wt[0] = 1.0 - wt[1];
    } else if (xa >= (double)n - 0.5) {   /* node n-1 at n-0.5 .. wall at n (value 0) */
        idx[0] = n - 1; idx[1] = -1;
        wt[1] = (xa - ((double)n - 0.5)) / 0.5; wt[0] = 1.0 - wt[1];
    } else {
        double s = xa - 0.5;
        double fl = floor(s);
        double w = s - fl;
        idx[0] = (long long)fl;
        idx[1] = idx[0] + 1;
        if (idx[1] > n - 1) idx[1] = n - 1;
        wt[0] = 1.0 - w;
        wt[1] = w;
    }
}

static void trilinear(const orc_t* o, const double* ufield, const double x[3], double u[3])
{
    long long ix[2], iy[2], iz[2];
    double wx[2], wy[2], wz[2];
    axis_stencil(o, 0, x[0], ix, wx);
    axis_stencil(o, 1, x[1], iy, wy);
    axis_stencil(o, 2, x[2], iz, wz);
    u[0] = u[1] = u[2] = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                if (ix[a] < 0 || iy[b] < 0 || iz[c] < 0) continue;   /* wall value 0 */
                double w = wx[a] * wy[b] * wz[c];
                long long cell = cell_index(o, ix[a], iy[b], iz[c]);
                for (int d = 0; d < 3; ++d) u[d] += w * ufield[3 * cell + d];
            }
}

/* Specular reflection at the no-slip walls (the walls bound the solute too). Returns 0 if
 * the point could not be brought back inside [0, n] on a walled axis. */
static int wall_reflect(const orc_t* o, double x[3])
{
    int ok = 1;
    for (int a = 0; a < 3; ++a) {
        if (!o->wall[a]) continue;
        double n = (double)o->n[a];
        for (int it = 0; it < 8; ++it) {
            if (x[a] < 0.0) x[a] = -x[a];
            else if (x[a] > n) x[a] = 2.0 * n - x[a];
            else break;
        }
        if (x[a] < 0.0 || x[a] > n) {
            ok = 0;
            x[a] = x[a] < 0.0 ? 0.0 : n;
        }
    }
    return ok;
}

static int beyond_wall(const orc_t* o, const double x[3])
{
    for (int a = 0; a < 3; ++a)
        if (o->wall[a] && (x[a] < 0.0 || x[a] > (double)o->n[a])) return 1;
    return 0;
}

static double f_at(const orc_t* o, const frame_t* fr, int p, const double xin[3], double g[3])
{
    double x[3] = {xin[0], xin[1], xin[2]};
    wrap_point(o, x);
    return metaball64(o, fr, p, x, g);
}

/* Algorithm 1: bisection on the segment from an outside point a (f < 1) to an inside point
 * b (f >= 1) of particle p. Convergence when |f(mid) - 1| < 1e-3; at most 200 iterations;
 * on f(mid) < 1 the outside end moves to mid, otherwise the inside end does. Returns 1 and
 * the point in xi on success, 0 when no such point was found (the error of Algorithm 1).
 * a_out receives the final outside end of the bracket. */
static int bisect(const orc_t* o, const frame_t* fr, int p, const double a_in[3], const double b_in[3],
                  double xi[3], double a_out[3])
{
    double a[3] = {a_in[0], a_in[1], a_in[2]}, b[3] = {b_in[0], b_in[1], b_in[2]};
    int found = 0;
    for (int it = 1; it <= 200; ++it) {
        double mid[3];
        for (int d = 0; d < 3; ++d) mid[d] = 0.5 * (a[d] + b[d]);
        double fm = f_at(o, fr, p, mid, NULL);
        if (fabs(fm - 1.0) < 1e-3) {
            for (int d = 0; d < 3; ++d) xi[d] = mid[d];
            found = 1;
            break;
        } else if (fm < 1.0) {
            for (int d = 0; d < 3; ++d) a[d] = mid[d];
        } else {
            for (int d = 0; d < 3; ++d) b[d] = mid[d];
        }
    }
    if (a_out) for (int d = 0; d < 3; ++d) a_out[d] = a[d];
    return found;
}

/* Algorithm 2 / Eqs. 18-22: t_o = x_int - x_p, t_i = x_f - x_int, n = grad f(x_int),
 * t_r = t_i - 2 (t_i . n) n. Reading: n is normalised (Eq. 22 is a mirror only for unit n).
 * Returns the reflected end point x_int + t_r. */
static void reflect(const orc_t* o, const frame_t* fr, int p, const double xint[3], const double xf[3],
                    double xnew[3])
{
    double g[3];
    f_at(o, fr, p, xint, g);
    double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double n[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
    double ti[3] = {xf[0] - xint[0], xf[1] - xint[1], xf[2] - xint[2]};
    double tn = ti[0] * n[0] + ti[1] * n[1] + ti[2] * n[2];
    for (int d = 0; d < 3; ++d) xnew[d] = xint[d] + (ti[d] - 2.0 * tn * n[d]);
}

/* Section 2.4.2 Dirichlet "refill" of a type-II walker at x inside particle p. Reading:
 *  1. s = -grad f / |grad f| at x (outward: Eq. 3 falls away from the control points);
 *  2. step out along s by h = 1/2, 1, 2, ..., 64 until f < 1 (bracket), then Algorithm 1 on
 *     [outside point, x] gives the surface point x_s;
 *  3. place the walker uniformly in the ball of radius sqrt(2 D dt) about x_s, from three
 *     uniforms of Philox counter (id, t, 1, 0): cos(theta) = 2U0 - 1, phi = 2 pi U1,
 *     r = R U2^(1/3); walls reflect it;
 *  4. if that point is inside a particle, mirror it across the tangent plane at x_s (outward
 *     normal of step 1 at x_s); if still inside, use the bracket's final outside end.
 * Returns 0 when step 2 or the final point failed (counted as a refill failure). */
static int refill(orc_t* o, const frame_t* fr, int p, const double x[3], uint32_t id, uint32_t t,
                  double xnew[3])
{
    double g[3];
    f_at(o, fr, p, x, g);
    double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double s[3] = {1.0, 0.0, 0.0};
    if (gn > 0.0 && isfinite(gn)) for (int d = 0; d < 3; ++d) s[d] = -g[d] / gn;
    double xo[3];
    int out = 0;
    for (double h = 0.5; h <= 64.0; h *= 2.0) {
        for (int d = 0; d < 3; ++d) xo[d] = x[d] + h * s[d];
        if (f_at(o, fr, p, xo, NULL) < 1.0) { out = 1; break; }
    }
    if (!out) { for (int d = 0; d < 3; ++d) xnew[d] = x[d]; return 0; }
    double xs[3], aend[3];
    if (!bisect(o, fr, p, xo, x, xs, aend)) {
        for (int d = 0; d < 3; ++d) xs[d] = aend[d];
    }
    double gs[3];
    f_at(o, fr, p, xs, gs);
    double gsn = sqrt(gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]);
    double nout[3] = {-gs[0] / gsn, -gs[1] / gsn, -gs[2] / gsn};
    uint32_t ctr[4] = {id, t, 1u, 0u}, r[4];
    philox4x32_10(o->key0, o->key1, ctr, r);
    double ct = 2.0 * u24(r[0]) - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * M_PI * u24(r[1]);
    double rad = sqrt(2.0 * o->D) * cbrt(u24(r[2]));
    double xr[3] = {xs[0] + rad * st * cos(ph), xs[1] + rad * st * sin(ph), xs[2] + rad * ct};
    wall_reflect(o, xr);
    if (inside_any64(o, fr, xr) >= 0) {
        double dn = (xr[0] - xs[0]) * nout[0] + (xr[1] - xs[1]) * nout[1] + (xr[2] - xs[2]) * nout[2];
        if (dn < 0.0) for (int d = 0; d < 3; ++d) xr[d] -= 2.0 * dn * nout[d];
        wall_reflect(o, xr);
        if (inside_any64(o, fr, xr) >= 0) {
            for (int d = 0; d < 3; ++d) xr[d] = aend[d];
            if (inside_any64(o, fr, xr) >= 0) {
                for (int d = 0; d < 3; ++d) xnew[d] = xr[d];
                return 0;
            }
        }
    }
    for (int d = 0; d < 3; ++d) xnew[d] = xr[d];
    return 1;
}

/* One walker, step t -> t+1 (Eq. 2 with dt = 1, then the rules of Section 2.4.2), velocity
 * field ufield of step t, particle frame fr1 at t+1. Types: I out/out and III in/out move
 * freely; II in/in is refilled; IV out/in is reflected by Algorithms 1 and 2, and a
 * reflected point that lands inside a particle or beyond a wall returns the walker to x
 * ("multiple reflections" in Section 2.4.2). */
static void walker_advance(orc_t* o, const frame_t* fr1, const double* ufield, uint32_t id, uint32_t t,
                           const double x[3], double xnew[3])
{
    double u[3];
    trilinear(o, ufield, x, u);
    uint32_t ctr[4] = {id, t, 0u, 0u}, r[4];
    philox4x32_10(o->key0, o->key1, ctr, r);
    double z[3];
    box_muller(u24(r[0]), u24(r[1]), &z[0], &z[1]);
    box_muller(u24(r[2]), u24(r[3]), &z[2], NULL);
    double amp = sqrt(2.0 * o->D * 1.0);
    double xf[3];
    for (int d = 0; d < 3; ++d) xf[d] = x[d] + u[d] * 1.0 + amp * z[d];
    if (!wall_reflect(o, xf)) o->wall_fail++;
    int pin = o->P ? inside_any64(o, fr1, x) : -1;
    int qin = o->P ? inside_any64(o, fr1, xf) : -1;
    if (pin >= 0 && qin >= 0) {                 /* type II: Dirichlet refill */
        o->cnt_type[1]++;
        if (!refill(o, fr1, pin, x, id, t, xnew)) o->refill_fail++;
    } else if (pin >= 0) {                      /* type III: moves out freely */
        o->cnt_type[2]++;
        for (int d = 0; d < 3; ++d) xnew[d] = xf[d];
    } else if (qin >= 0) {                      /* type IV: no-flux reflection */
        o->cnt_type[3]++;
        double xi[3], tr[3];
        if (!bisect(o, fr1, qin, x, xf, xi, NULL)) {
            o->bisect_fail++;                   /* Reading: the walker stays where it was */
            for (int d = 0; d < 3; ++d) xnew[d] = x[d];
            return;
        }
        reflect(o, fr1, qin, xi, xf, tr);
        if (beyond_wall(o, tr) || inside_any64(o, fr1, tr) >= 0) {
            for (int d = 0; d < 3; ++d) xnew[d] = x[d];
        } else {
            for (int d = 0; d < 3; ++d) xnew[d] = tr[d];
        }
    } else {                                    /* type I */
        o->cnt_type[0]++;
        for (int d = 0; d < 3; ++d) xnew[d] = xf[d];
    }
}

static void walkers_step(orc_t* o, long long t)
{
    if (o->nw == 0) return;
    frame_t fr1;
    frame_alloc(o, &fr1);
    frame_at(o, t + 1, &fr1);
    for (long long w = 0; w < o->nw; ++w) {
        double xn[3];
        walker_advance(o, &fr1, o->u, (uint32_t)w, (uint32_t)t, o->x + 3 * w, xn);
        for (int d = 0; d < 3; ++d) o->x[3 * w + d] = xn[d];
    }
    frame_free(&fr1);
}

/* Eq. 16 bins walkers by the cell that holds them: n_s(x, t). Positions are unwrapped;
 * periodic axes wrap, walled axes clamp x = n into the last cell. */
static long long walker_cell(const orc_t* o, const double x[3])
{
    long long c[3];
    for (int a = 0; a < 3; ++a) {
        long long i = (long long)floor(x[a]);
        if (o->wall[a]) { if (i < 0) i = 0; if (i > o->n[a] - 1) i = o->n[a] - 1; }
        else i = wrapll(i, o->n[a]);
        c[a] = i;
    }
    return cell_index(o, c[0], c[1], c[2]);
}

/* ------------------------------------------------------------------------------------------
 * Free DEM (Section 2.2, Eqs. 4-11), used instead of the prescribed trajectories once
 * orc_set_dem has been called. Units are lattice units; one LBM step holds `substeps` DEM
 * steps of dt = 1 / substeps. Readings (the paper leaves these open or defers them to its
 * references):
 *  - Sphero-metaball (Eq. 6 context): particle p's contact shape is its metaball scaled about the
 *    body origin by s_p = 1 - R_s,p / R_c,p (control points times s_p, weights times s_p^2) and
 *    dilated by the sphere radius R_s,p, with R_c,p = max_i (|c_i| + sqrt(k_i)) over the
 *    body-frame control points, so a single centre at the origin is reproduced exactly. The
 *    bound radius R_b,p (f_p < 1 beyond it) only skips pairs and faces out of reach.
 *  - Pair contact (Eqs. 6-9): Newton-Raphson on grad(f0 + f1) = 0 (Eq. 7) for the internal
 *    metaballs, at most DEM_NEWTON_NEW iterations from the deterministic start below, or
 *    DEM_NEWTON_CONT from the previous DEM step's point while the contact lasts; a step longer
 *    than one lattice unit is scaled to one, and a singular Hessian or a step below 1e-12 ends
 *    the iteration. Pairs and faces out of reach (bound spheres apart) are skipped: they cannot
 *    touch, so skipping changes no result.
 *    Eq. 8: q0 is chosen so that f0(x_m + q0 grad f0(x_m)) = 1 holds, as the text imposes:
 *    the crossing nearest to x_m, from the printed first-order Taylor value by a bracketed
 *    Newton iteration in q0 (surface_along). The single first-order step misplaces the surface
 *    point by about a lattice unit when x_m lies far from it, which happens when R_s is
 *    comparable to the gap between the internal shapes. Eq. 9 with
 *    n = (x_c1 - x_c0) / |x_c1 - x_c0| from particle 0 towards particle 1 and
 *    x_cp = x_c0 + (R_s0 - delta/2) n, the middle of the overlap (the printed orientation of n
 *    would put the contact point inside particle 0).
 *    Start: the internal control points a of particle 0 and b of particle 1 with the smallest
 *    |c_a - c_b| - r_a - r_b (r = sqrt of the internal weight; first pair on ties), and
 *    x = c_a + r_a / (r_a + r_b) (c_b - c_a).
 *  - Wall contact (Eqs. 10-11) on both faces of every walled axis: Newton-Raphson on
 *    (d_b f, d_c f, f - 1) = 0 (b, c the two axes along the face) gives the point x_cm of the
 *    internal surface closest to the face; x_cw is its projection on the face, n the face's
 *    normal into the box, delta = R_s - (x_cm - x_cw).n, x_cp = x_cw + delta/2 n as printed.
 *    Start: the control point reaching farthest towards the face, moved by its internal radius.
 *  - Normal force (linear spring-dashpot): F_n = max(0, k_n delta + eta_n (v_i - v_j).n_ij),
 *    with n_ij from particle i towards the other body and velocities taken at the contact point;
 *    it acts on i along -n_ij (no attraction).
 *  - Tangential force (Eq. 5): the spring xi, projected on the current tangent plane, grows by
 *    v_t dt (v_t: tangential part of the other body's contact-point velocity relative to i's);
 *    F_t0 = k_t xi + eta_t v_t on i; when |F_t0| > mu_s F_n the force is mu_s F_n F_t0/|F_t0|
 *    and the spring is reset to (F_t - eta_t v_t) / k_t. The spring is cleared when the contact
 *    ends.
 *  - Eq. 4, per DEM step: F = m g + sum F^c + F^e, T = sum T^c + T^e (torques about the
 *    origin); v += dt F / m, o += dt v (symplectic Euler); w += dt I_w^-1 (T - w x I_w w) with
 *    I_w = R I_b R^T; q += dt/2 (0, w) q, then normalised. F^e and T^e are the hydrodynamic
 *    force and torque of the LBM update of the same step, held over its DEM steps (or zero
 *    with the hydrodynamic coupling off). Pair forces are summed per particle in pair order,
 *    then the wall forces.
 *  - Periodic axes: a pair is evaluated at the minimum image of the second origin relative to
 *    the first; origins stay unwrapped.
 * ------------------------------------------------------------------------------------------ */
#define DEM_NEWTON_NEW 24
#define DEM_NEWTON_CONT 6
#define DEM_SURFACE_ITERS 24
#define DEM_SURFACE_HALVINGS 16

/* Rotation matrix of the unit quaternion (w, x, y, z) */
static void quat_matrix(const double* q, double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
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

static void dem_pose(const orc_t* o, int p, double org[3], double vel[3], double R[3][3])
{
    const double* st = o->dst + 13 * (size_t)p;
    for (int a = 0; a < 3; ++a) { org[a] = st[a]; vel[a] = st[7 + a]; }
    quat_matrix(st + 3, R);
}

/* Internal (zoomed) control points of particle p in world coordinates about origin org, and
 * their weights; returns their count */
static int dem_internal(const orc_t* o, int p, const double org[3], double* cw, double* kw)
{
    double R[3][3], dummy[3], od[3];
    dem_pose(o, p, od, dummy, R);
    double s = o->dzoom[p];
    int n = 0;
    for (int i = o->coff[p]; i < o->coff[p + 1]; ++i, ++n) {
        double b[3] = {s * o->cbody[3 * i], s * o->cbody[3 * i + 1], s * o->cbody[3 * i + 2]};
        for (int a = 0; a < 3; ++a) cw[3 * n + a] = org[a] + R[a][0] * b[0] + R[a][1] * b[1] + R[a][2] * b[2];
        kw[n] = s * s * o->kc[i];
    }
    return n;
}

/* Eq. 3 with its gradient and Hessian (xx yy zz xy xz yz) at x, no wrapping */
static double mb_eval(const double* cw, const double* kw, int n, const double x[3], double g[3], double H[6])
{
    double f = 0.0;
    for (int a = 0; a < 3; ++a) g[a] = 0.0;
    for (int m = 0; m < 6; ++m) H[m] = 0.0;
    for (int i = 0; i < n; ++i) {
        double r[3] = {x[0] - cw[3 * i], x[1] - cw[3 * i + 1], x[2] - cw[3 * i + 2]};
        double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        double inv2 = 1.0 / r2, k = kw[i];
        double fi = k * inv2;
        f += fi;
        double c1 = -2.0 * fi * inv2;          /* d/dx k/r^2 = -2 k r / r^4 */
        double c2 = 8.0 * fi * inv2 * inv2;    /* second derivative: -2k/r^4 I + 8k r r^T / r^6 */
        for (int a = 0; a < 3; ++a) g[a] += c1 * r[a];
        H[0] += c1 + c2 * r[0] * r[0];
        H[1] += c1 + c2 * r[1] * r[1];
        H[2] += c1 + c2 * r[2] * r[2];
        H[3] += c2 * r[0] * r[1];
        H[4] += c2 * r[0] * r[2];
        H[5] += c2 * r[1] * r[2];
    }
    return f;
}

/* Solves the 3x3 system A d = b by Cramer's rule; returns 0 when |det| is tiny */
static int solve3(double A[3][3], const double b[3], double d[3])
{
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(fabs(det) > 1e-300)) return 0;
    d[0] = (b[0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (b[1] * A[2][2] - A[1][2] * b[2])
            + A[0][2] * (b[1] * A[2][1] - A[1][1] * b[2])) / det;
    d[1] = (A[0][0] * (b[1] * A[2][2] - A[1][2] * b[2]) - b[0] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
            + A[0][2] * (A[1][0] * b[2] - b[1] * A[2][0])) / det;
    d[2] = (A[0][0] * (A[1][1] * b[2] - b[1] * A[2][1]) - A[0][1] * (A[1][0] * b[2] - b[1] * A[2][0])
            + b[0] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / det;
    return 1;
}

/* Newton step with its length limited to one lattice unit; returns 0 when singular or when the
 * step was below 1e-12 (converged) */
static int newton_update(double A[3][3], const double G[3], double x[3])
{
    double b[3] = {-G[0], -G[1], -G[2]}, d[3];
    if (!solve3(A, b, d)) return 0;
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double sc = len > 1.0 ? 1.0 / len : 1.0;
    for (int a = 0; a < 3; ++a) x[a] += sc * d[a];
    return len > 1e-12;
}

/* Eq. 8: x_c = x_m + q grad f(x_m) with f(x_c) = 1, the crossing nearest to x_m. q starts from
 * the printed first-order Taylor value q1 = (1 - f(x_m)) / |grad f(x_m)|^2; the bracket is
 * [0, q_in] with q_in the first of q1, q1/2, q1/4, ... (at most DEM_SURFACE_HALVINGS halvings)
 * where f >= 1; then DEM_SURFACE_ITERS Newton steps in q (each the same Taylor step from the
 * current point), a step that leaves the bracket replaced by bisection. Without an inside point
 * q stays q1. */
static void surface_along(const double* c, const double* k, int n, const double xm[3], double xc[3])
{
    double g[3], gx[3], H[6], x[3];
    double f = mb_eval(c, k, n, xm, g, H);
    double q1 = (1.0 - f) / (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    double lo = 0.0, hi = q1, q = q1;
    int inside = 0;
    for (int h = 0; h <= DEM_SURFACE_HALVINGS; ++h) {
        for (int a = 0; a < 3; ++a) x[a] = xm[a] + hi * g[a];
        if (mb_eval(c, k, n, x, gx, H) >= 1.0) { inside = 1; break; }
        hi = 0.5 * hi;
    }
    if (inside) {
        q = hi;
        for (int it = 0; it < DEM_SURFACE_ITERS; ++it) {
            for (int a = 0; a < 3; ++a) x[a] = xm[a] + q * g[a];
            double fx = mb_eval(c, k, n, x, gx, H);
            if (fx == 1.0) break;
            if (fx > 1.0) hi = q; else lo = q;
            double dq = gx[0] * g[0] + gx[1] * g[1] + gx[2] * g[2];
            double qn = fabs(dq) > 1e-300 ? q - (fx - 1.0) / dq : 0.5 * (lo + hi);
            if (!(qn > lo && qn < hi)) qn = 0.5 * (lo + hi);
            if (qn == q) break;
            q = qn;
        }
    }
    for (int a = 0; a < 3; ++a) xc[a] = xm[a] + q * g[a];
}

/* Contact geometry of one pair (Eqs. 7-9). xm: in = start (when cont), out = Newton point.
 * Returns delta; writes x_c0, x_c1, n (0 towards 1) and x_cp. */
static double dem_pair_geom(const double* c0, const double* k0, int n0, const double* c1, const double* k1,
                            int n1, double Rs0, double Rs1, int cont, double xm[3], double xc0[3],
                            double xc1[3], double nrm[3], double xcp[3])
{
    if (!cont) {
        int ba = 0, bb = 0;
        double best = INFINITY;
        for (int a = 0; a < n0; ++a)
            for (int b = 0; b < n1; ++b) {
                double d[3] = {c1[3 * b] - c0[3 * a], c1[3 * b + 1] - c0[3 * a + 1], c1[3 * b + 2] - c0[3 * a + 2]};
                double gap = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - sqrt(k0[a]) - sqrt(k1[b]);
                if (gap < best) { best = gap; ba = a; bb = b; }
            }
        double ra = sqrt(k0[ba]), rb = sqrt(k1[bb]), w = ra / (ra + rb);
        for (int a = 0; a < 3; ++a) xm[a] = c0[3 * ba + a] + w * (c1[3 * bb + a] - c0[3 * ba + a]);
    }
    int iters = cont ? DEM_NEWTON_CONT : DEM_NEWTON_NEW;
    for (int it = 0; it < iters; ++it) {
        double g0[3], g1[3], H0[6], H1[6];
        mb_eval(c0, k0, n0, xm, g0, H0);
        mb_eval(c1, k1, n1, xm, g1, H1);
        double G[3] = {g0[0] + g1[0], g0[1] + g1[1], g0[2] + g1[2]};
        double A[3][3] = {{H0[0] + H1[0], H0[3] + H1[3], H0[4] + H1[4]},
                          {H0[3] + H1[3], H0[1] + H1[1], H0[5] + H1[5]},
                          {H0[4] + H1[4], H0[5] + H1[5], H0[2] + H1[2]}};
        if (!newton_update(A, G, xm)) break;
    }
    surface_along(c0, k0, n0, xm, xc0);
    surface_along(c1, k1, n1, xm, xc1);
    double d[3] = {xc1[0] - xc0[0], xc1[1] - xc0[1], xc1[2] - xc0[2]};
    double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double delta = Rs0 + Rs1 - dist;
    for (int a = 0; a < 3; ++a) nrm[a] = dist > 0.0 ? d[a] / dist : 0.0;
    for (int a = 0; a < 3; ++a) xcp[a] = xc0[a] + (Rs0 - 0.5 * delta) * nrm[a];
    return delta;
}

/* Contact geometry of a particle and the face `side` (0: plane x_a = 0, 1: plane x_a = L) of
 * walled axis a (Eqs. 10-11). Returns delta; writes x_cm, x_cw, n (into the box), x_cp. */
static double dem_wall_geom(const double* c, const double* k, int n, int a, int side, double L, double Rs,
                            int cont, double xm[3], double xcw[3], double nrm[3], double xcp[3])
{
    double sg = side ? -1.0 : 1.0;   /* inward normal along axis a */
    if (!cont) {
        int bi = 0;
        double best = INFINITY;
        for (int i = 0; i < n; ++i) {
            double reach = side ? -(c[3 * i + a] + sqrt(k[i])) : c[3 * i + a] - sqrt(k[i]);
            if (reach < best) { best = reach; bi = i; }
        }
        for (int b = 0; b < 3; ++b) xm[b] = c[3 * bi + b];
        xm[a] -= sg * sqrt(k[bi]);
    }
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    if (b > cc) { int t = b; b = cc; cc = t; }
    int iters = cont ? DEM_NEWTON_CONT : DEM_NEWTON_NEW;
    for (int it = 0; it < iters; ++it) {
        double g[3], H6[6];
        double f = mb_eval(c, k, n, xm, g, H6);
        double H[3][3] = {{H6[0], H6[3], H6[4]}, {H6[3], H6[1], H6[5]}, {H6[4], H6[5], H6[2]}};
        double G[3] = {g[b], g[cc], f - 1.0};
        double A[3][3] = {{H[b][0], H[b][1], H[b][2]}, {H[cc][0], H[cc][1], H[cc][2]}, {g[0], g[1], g[2]}};
        if (!newton_update(A, G, xm)) break;
    }
    for (int d = 0; d < 3; ++d) { xcw[d] = xm[d]; nrm[d] = 0.0; }
    xcw[a] = side ? L : 0.0;
    nrm[a] = sg;
    double dist = (xm[a] - xcw[a]) * sg;
    double delta = Rs - dist;
    for (int d = 0; d < 3; ++d) xcp[d] = xcw[d] + 0.5 * delta * nrm[d];
    return delta;
}

/* Velocity of body p's material point at x (origin org): v + w x (x - org) */
static void dem_point_velocity(const orc_t* o, int p, const double org[3], const double x[3], double v[3])
{
    const double* st = o->dst + 13 * (size_t)p;
    double r[3] = {x[0] - org[0], x[1] - org[1], x[2] - org[2]};
    const double* w = st + 10;
    v[0] = st[7] + (w[1] * r[2] - w[2] * r[1]);
    v[1] = st[8] + (w[2] * r[0] - w[0] * r[2]);
    v[2] = st[9] + (w[0] * r[1] - w[1] * r[0]);
}

/* Contact force on body i (normal spring-dashpot and Eq. 5). n: from i towards the other body;
 * vi, vj: contact-point velocities; xi: the contact's tangential spring, updated. */
static void dem_contact_force(const orc_t* o, double delta, const double n[3], const double vi[3],
                              const double vj[3], double dt, double xi[3], double F[3])
{
    double vr[3] = {vj[0] - vi[0], vj[1] - vi[1], vj[2] - vi[2]};
    double vn = vr[0] * n[0] + vr[1] * n[1] + vr[2] * n[2];   /* -(v_i - v_j).n */
    double Fn = o->dem_kn * delta - o->dem_etan * vn;
    if (Fn < 0.0) Fn = 0.0;
    double vt[3] = {vr[0] - vn * n[0], vr[1] - vn * n[1], vr[2] - vn * n[2]};
    double xn = xi[0] * n[0] + xi[1] * n[1] + xi[2] * n[2];
    for (int a = 0; a < 3; ++a) xi[a] = (xi[a] - xn * n[a]) + vt[a] * dt;
    double Ft[3];
    for (int a = 0; a < 3; ++a) Ft[a] = o->dem_kt * xi[a] + o->dem_etat * vt[a];
    double mag = sqrt(Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2]);
    double lim = o->dem_mus * Fn;
    if (mag > lim) {
        double sc = lim / mag;
        for (int a = 0; a < 3; ++a) {
            Ft[a] = Ft[a] * sc;
            xi[a] = o->dem_kt > 0.0 ? (Ft[a] - o->dem_etat * vt[a]) / o->dem_kt : 0.0;
        }
    }
    for (int a = 0; a < 3; ++a) F[a] = Ft[a] - Fn * n[a];
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Minimum-image origin of particle j seen from particle i's origin (origins unwrapped) */
static void dem_image(const orc_t* o, const double oi[3], const double oj[3], double out[3])
{
    for (int a = 0; a < 3; ++a) {
        double d = oj[a] - oi[a];
        if (!o->wall[a]) d -= (double)o->n[a] * floor(d / (double)o->n[a] + 0.5);
        out[a] = oi[a] + d;
    }
}

/* Pair (i < j) force and torques of one DEM step, from the state at its start; updates the
 * pair's spring, Newton point and contact flag. Writes the force on i and both torques. */
static void dem_pair(orc_t* o, int i, int j, double dt, double Fi[3], double Ti[3], double Tj[3],
                     double* cbuf, double* kbuf)
{
    size_t pr = (size_t)i * o->P + j;
    for (int a = 0; a < 3; ++a) Fi[a] = Ti[a] = Tj[a] = 0.0;
    const double* si = o->dst + 13 * (size_t)i;
    const double* sj = o->dst + 13 * (size_t)j;
    double oj[3];
    dem_image(o, si, sj, oj);
    double d[3] = {oj[0] - si[0], oj[1] - si[1], oj[2] - si[2]};
    double reach = o->Rb[i] + o->Rb[j];
    if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] >= reach * reach) {   /* bound spheres apart */
        o->dact[pr] = 0;
        for (int a = 0; a < 3; ++a) o->dxi[3 * pr + a] = 0.0;
        return;
    }
    double* c0 = cbuf; double* k0 = kbuf;
    int n0 = dem_internal(o, i, si, c0, k0);
    double* c1 = cbuf + 3 * n0; double* k1 = kbuf + n0;
    int n1 = dem_internal(o, j, oj, c1, k1);
    double xc0[3], xc1[3], nrm[3], xcp[3];
    double* xm = o->dxm + 3 * pr;
    double delta = dem_pair_geom(c0, k0, n0, c1, k1, n1, o->dRs[i], o->dRs[j], o->dact[pr] != 0, xm, xc0, xc1,
                                 nrm, xcp);
    double* xi = o->dxi + 3 * pr;
    if (!(delta > 0.0)) {
        o->dact[pr] = 0;
        for (int a = 0; a < 3; ++a) xi[a] = 0.0;
        return;
    }
    o->dact[pr] = 1;
    double vi[3], vj[3];
    dem_point_velocity(o, i, si, xcp, vi);
    dem_point_velocity(o, j, oj, xcp, vj);
    dem_contact_force(o, delta, nrm, vi, vj, dt, xi, Fi);
    double ri[3] = {xcp[0] - si[0], xcp[1] - si[1], xcp[2] - si[2]};
    double rj[3] = {xcp[0] - oj[0], xcp[1] - oj[1], xcp[2] - oj[2]};
    double Fj[3] = {-Fi[0], -Fi[1], -Fi[2]};
    cross3(ri, Fi, Ti);
    cross3(rj, Fj, Tj);
}

/* Wall face f = 2 a + side of particle p: force and torque of one DEM step */
static void dem_wall(orc_t* o, int p, int f, double dt, double Fw[3], double Tw[3], double* cbuf, double* kbuf)
{
    size_t wi = 6 * (size_t)p + f;
    int a = f >> 1, side = f & 1;
    for (int b = 0; b < 3; ++b) Fw[b] = Tw[b] = 0.0;
    const double* sp = o->dst + 13 * (size_t)p;
    double L = (double)o->n[a];
    double gap = side ? L - sp[a] : sp[a];
    if (!o->wall[a] || gap >= o->Rb[p]) {
        o->dactw[wi] = 0;
        for (int b = 0; b < 3; ++b) o->dxiw[3 * wi + b] = 0.0;
        return;
    }
    int n = dem_internal(o, p, sp, cbuf, kbuf);
    double xcw[3], nrm[3], xcp[3];
    double* xm = o->dxmw + 3 * wi;
    double delta = dem_wall_geom(cbuf, kbuf, n, a, side, L, o->dRs[p], o->dactw[wi] != 0, xm, xcw, nrm, xcp);
    double* xi = o->dxiw + 3 * wi;
    if (!(delta > 0.0)) {
        o->dactw[wi] = 0;
        for (int b = 0; b < 3; ++b) xi[b] = 0.0;
        return;
    }
    o->dactw[wi] = 1;
    double vi[3], vw[3] = {0.0, 0.0, 0.0};
    dem_point_velocity(o, p, sp, xcp, vi);
    double nw[3] = {-nrm[0], -nrm[1], -nrm[2]};   /* from the particle towards the wall */
    dem_contact_force(o, delta, nw, vi, vw, dt, xi, Fw);
    double r[3] = {xcp[0] - sp[0], xcp[1] - sp[1], xcp[2] - sp[2]};
    cross3(r, Fw, Tw);
}

/* One DEM step of length dt (Eq. 4) with hydrodynamic force Fe, torque Te (may be NULL) */
static void dem_substep(orc_t* o, double dt, const double* Fe, const double* Te)
{
    int P = o->P;
    size_t PP = (size_t)P * P;
    double* pF = (double*)calloc(3 * PP + 3, sizeof(double));
    double* pTi = (double*)calloc(3 * PP + 3, sizeof(double));
    double* pTj = (double*)calloc(3 * PP + 3, sizeof(double));
    double* wF = (double*)calloc(18 * (size_t)P + 3, sizeof(double));
    double* wT = (double*)calloc(18 * (size_t)P + 3, sizeof(double));
    double* cbuf = (double*)malloc(sizeof(double) * (6 * (size_t)o->Nc + 6));
    double* kbuf = (double*)malloc(sizeof(double) * (2 * (size_t)o->Nc + 2));
    for (int i = 0; i < P; ++i)
        for (int j = i + 1; j < P; ++j) {
            size_t pr = (size_t)i * P + j;
            dem_pair(o, i, j, dt, pF + 3 * pr, pTi + 3 * pr, pTj + 3 * pr, cbuf, kbuf);
        }
    for (int p = 0; p < P; ++p)
        for (int f = 0; f < 6; ++f) dem_wall(o, p, f, dt, wF + 3 * (6 * (size_t)p + f), wT + 3 * (6 * (size_t)p + f), cbuf, kbuf);
    for (int p = 0; p < P; ++p) {
        double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < P; ++j) {
            if (j < p) {
                size_t pr = (size_t)j * P + p;
                for (int a = 0; a < 3; ++a) { F[a] = F[a] - pF[3 * pr + a]; T[a] = T[a] + pTj[3 * pr + a]; }
            } else if (j > p) {
                size_t pr = (size_t)p * P + j;
                for (int a = 0; a < 3; ++a) { F[a] = F[a] + pF[3 * pr + a]; T[a] = T[a] + pTi[3 * pr + a]; }
            }
        }
        for (int f = 0; f < 6; ++f)
            for (int a = 0; a < 3; ++a) {
                F[a] = F[a] + wF[3 * (6 * (size_t)p + f) + a];
                T[a] = T[a] + wT[3 * (6 * (size_t)p + f) + a];
            }
        double m = o->dmass[p];
        for (int a = 0; a < 3; ++a) {
            if (Fe) { F[a] = F[a] + Fe[3 * p + a]; T[a] = T[a] + Te[3 * p + a]; }
            F[a] = F[a] + m * o->dem_g[a];
        }
        double* st = o->dst + 13 * (size_t)p;
        /* translation: symplectic Euler */
        for (int a = 0; a < 3; ++a) {
            st[7 + a] = st[7 + a] + dt * (F[a] / m);
            st[a] = st[a] + dt * st[7 + a];
        }
        /* rotation: I_w = R I_b R^T, w += dt I_w^-1 (T - w x I_w w) */
        double R[3][3];
        quat_matrix(st + 3, R);
        const double* Ib6 = o->dIb + 6 * (size_t)p;
        double Ib[3][3] = {{Ib6[0], Ib6[3], Ib6[4]}, {Ib6[3], Ib6[1], Ib6[5]}, {Ib6[4], Ib6[5], Ib6[2]}};
        double RI[3][3], Iw[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) RI[a][b] = R[a][0] * Ib[0][b] + R[a][1] * Ib[1][b] + R[a][2] * Ib[2][b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Iw[a][b] = RI[a][0] * R[b][0] + RI[a][1] * R[b][1] + RI[a][2] * R[b][2];
        double* w = st + 10;
        double Lw[3] = {Iw[0][0] * w[0] + Iw[0][1] * w[1] + Iw[0][2] * w[2],
                        Iw[1][0] * w[0] + Iw[1][1] * w[1] + Iw[1][2] * w[2],
                        Iw[2][0] * w[0] + Iw[2][1] * w[1] + Iw[2][2] * w[2]};
        double gyro[3];
        cross3(w, Lw, gyro);
        double rhs[3] = {T[0] - gyro[0], T[1] - gyro[1], T[2] - gyro[2]}, dw[3];
        if (solve3(Iw, rhs, dw))
            for (int a = 0; a < 3; ++a) w[a] = w[a] + dt * dw[a];
        /* orientation: q += dt/2 (0, w) q, normalised */
        double* q = st + 3;
        double qw = q[0], qv[3] = {q[1], q[2], q[3]}, wxq[3];
        cross3(w, qv, wxq);
        double h = 0.5 * dt;
        double nq[4] = {qw - h * (w[0] * qv[0] + w[1] * qv[1] + w[2] * qv[2]),
                        qv[0] + h * (qw * w[0] + wxq[0]),
                        qv[1] + h * (qw * w[1] + wxq[1]),
                        qv[2] + h * (qw * w[2] + wxq[2])};
        double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
        for (int a = 0; a < 4; ++a) q[a] = nq[a] / nn;
    }
    free(pF); free(pTi); free(pTj); free(wF); free(wT); free(cbuf); free(kbuf);
}

/* The DEM part of one LBM step: `substeps` DEM steps with the hydrodynamic force and torque of
 * the LBM update just made (Fp, Tp), when the coupling is on */
static void dem_advance(orc_t* o)
{
    double dt = 1.0 / (double)o->dem_nsub;
    for (int s = 0; s < o->dem_nsub; ++s)
        dem_substep(o, dt, o->dem_hydro ? o->Fp : NULL, o->dem_hydro ? o->Tp : NULL);
}

/* ------------------------------------------------------------------------------------------
 * Exported API (ctypes). All arrays are host arrays owned by the caller.
 * ------------------------------------------------------------------------------------------ */
ORC_API void* orc_create(const int dims[3], int q, double tau, double D, uint64_t seed,
                         int wall_mask, const double F0[3], double Fperiod, double rho0,
                         const double u_init[3])
{
    if (q != 15 && q != 19) return NULL;
    orc_t* o = (orc_t*)calloc(1, sizeof(orc_t));
    for (int a = 0; a < 3; ++a) {
        o->n[a] = dims[a];
        o->wall[a] = (wall_mask >> a) & 1;
        o->F0[a] = F0[a];
        o->u_init[a] = u_init[a];
    }
    o->ncell = (long long)dims[0] * dims[1] * dims[2];
    o->q = q; o->tau = tau; o->D = D;
    o->key0 = (uint32_t)seed; o->key1 = (uint32_t)(seed >> 32);
    o->Fperiod = Fperiod; o->rho0 = rho0;
    o->f = (double*)malloc(sizeof(double) * (size_t)q * o->ncell);
    o->fn = (double*)malloc(sizeof(double) * (size_t)q * o->ncell);
    o->u = (double*)calloc(3 * (size_t)o->ncell, sizeof(double));
    o->rho = (double*)calloc((size_t)o->ncell, sizeof(double));
    o->cnt = (int*)calloc((size_t)o->ncell, sizeof(int));
    o->own = (int*)malloc(sizeof(int) * (size_t)o->ncell);
    for (long long c = 0; c < o->ncell; ++c) o->own[c] = -1;
    o->solid_time = -1;
    /* initial state: equilibrium at rho0 and u_init (post-collision of step -1) */
    for (int m = 0; m < q; ++m) {
        double fe = feq(q, m, rho0, u_init);
        for (long long c = 0; c < o->ncell; ++c) o->f[(size_t)m * o->ncell + c] = fe;
    }
    for (long long c = 0; c < o->ncell; ++c) {
        o->rho[c] = rho0;
        for (int a = 0; a < 3; ++a) o->u[3 * c + a] = u_init[a];
    }
    o->coff = (int*)calloc(1, sizeof(int));
    return o;
}

ORC_API void orc_destroy(void* h)
{
    orc_t* o = (orc_t*)h;
    if (!o) return;
    free(o->f); free(o->fn); free(o->u); free(o->rho); free(o->cnt); free(o->own);
    free(o->coff); free(o->cbody); free(o->kc); free(o->kc32);
    free(o->org); free(o->amp); free(o->per); free(o->pha); free(o->omg); free(o->Rb);
    free(o->Fp); free(o->Tp); free(o->x); free(o->x0);
    free(o->dst); free(o->dmass); free(o->dIb); free(o->dRs); free(o->dzoom); free(o->dcm); free(o->dem_nodes);
    free(o->dxi); free(o->dxm); free(o->dact); free(o->dxiw); free(o->dxmw); free(o->dactw);
    free(o);
}

ORC_API int orc_set_metaballs(void* h, int P, const int* coff, const float* cbody, const float* k,
                              const double* origin, const double* amp, const double* per,
                              const double* pha, const double* omega)
{
    orc_t* o = (orc_t*)h;
    free(o->coff); free(o->cbody); free(o->kc); free(o->kc32);
    free(o->org); free(o->amp); free(o->per); free(o->pha); free(o->omg); free(o->Rb);
    free(o->Fp); free(o->Tp);
    o->P = P;
    o->Nc = coff[P];
    o->coff = (int*)malloc(sizeof(int) * (size_t)(P + 1));
    memcpy(o->coff, coff, sizeof(int) * (size_t)(P + 1));
    o->cbody = (double*)malloc(sizeof(double) * 3 * (size_t)o->Nc + 8);
    o->kc = (double*)malloc(sizeof(double) * (size_t)o->Nc + 8);
    o->kc32 = (float*)malloc(sizeof(float) * (size_t)o->Nc + 8);
    for (int i = 0; i < o->Nc; ++i) {
        for (int a = 0; a < 3; ++a) o->cbody[3 * i + a] = (double)cbody[3 * i + a];
        o->kc[i] = (double)k[i];
        o->kc32[i] = k[i];
    }
    size_t p3 = sizeof(double) * 3 * (size_t)P + 8, p1 = sizeof(double) * (size_t)P + 8;
    o->org = (double*)malloc(p3); o->amp = (double*)malloc(p3); o->omg = (double*)malloc(p3);
    o->per = (double*)malloc(p1); o->pha = (double*)malloc(p1); o->Rb = (double*)malloc(p1);
    o->Fp = (double*)calloc(3 * (size_t)P + 1, sizeof(double));
    o->Tp = (double*)calloc(3 * (size_t)P + 1, sizeof(double));
    for (int p = 0; p < P; ++p) {
        for (int a = 0; a < 3; ++a) {
            o->org[3 * p + a] = origin[3 * p + a];
            o->amp[3 * p + a] = amp[3 * p + a];
            o->omg[3 * p + a] = omega ? omega[3 * p + a] : 0.0;
        }
        o->per[p] = per[p];
        o->pha[p] = pha[p];
    }
    for (int p = 0; p < P; ++p) o->Rb[p] = bound_radius(o, p);
    o->solid_time = -1;
    return 0;
}

/* Seeding: walker w tries Philox counters (w, a, 2, 0), a = 0, 1, ..., taking three uniforms
 * as a point lo + U (hi - lo) of the seed box (FP64, rounded to binary32), and keeps the
 * first point outside every particle at the current time (binary32 test). Walkers that start
 * inside a particle are removed at the first step in Section 2.4.2; drawing again keeps the
 * requested count exact. Returns the number of walkers that found no free point. */
ORC_API long long orc_seed_walkers(void* h, long long n, const double lo[3], const double hi[3],
                                   int max_attempts)
{
    orc_t* o = (orc_t*)h;
    free(o->x); free(o->x0);
    o->nw = n;
    o->x = (double*)malloc(sizeof(double) * 3 * (size_t)n + 8);
    o->x0 = (double*)malloc(sizeof(double) * 3 * (size_t)n + 8);
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, o->t, &fr);
    long long fails = 0;
    for (long long w = 0; w < n; ++w) {
        float xs[3] = {0.0f, 0.0f, 0.0f};
        int ok = 0;
        for (int a = 0; a < max_attempts && !ok; ++a) {
            uint32_t ctr[4] = {(uint32_t)w, (uint32_t)a, 2u, 0u}, r[4];
            philox4x32_10(o->key0, o->key1, ctr, r);
            for (int d = 0; d < 3; ++d) {
                volatile double span = hi[d] - lo[d];
                volatile double off = u24(r[d]) * span;
                xs[d] = (float)(lo[d] + off);
            }
            ok = (o->P == 0) || inside_any32(o, &fr, xs) < 0;
        }
        if (!ok) fails++;
        for (int d = 0; d < 3; ++d) o->x[3 * w + d] = o->x0[3 * w + d] = (double)xs[d];
    }
    frame_free(&fr);
    o->seed_fail += fails;
    return fails;
}

ORC_API void orc_set_walkers(void* h, long long n, const double* x, const double* x0)
{
    orc_t* o = (orc_t*)h;
    free(o->x); free(o->x0);
    o->nw = n;
    o->x = (double*)malloc(sizeof(double) * 3 * (size_t)n + 8);
    o->x0 = (double*)malloc(sizeof(double) * 3 * (size_t)n + 8);
    memcpy(o->x, x, sizeof(double) * 3 * (size_t)n);
    memcpy(o->x0, x0 ? x0 : x, sizeof(double) * 3 * (size_t)n);
}

/* n timesteps: solid fraction at t, LBM at t, walkers t -> t+1 with the particles at t+1 */
ORC_API void orc_step(void* h, long long nsteps)
{
    orc_t* o = (orc_t*)h;
    for (long long s = 0; s < nsteps; ++s) {
        if (!o->coupling) rasterize(o, o->t);
        lbm_step(o, o->t);
        if (o->dem) dem_advance(o);   /* particles t -> t+1 with the force of this update */
        walkers_step(o, o->t);
        o->t++;
    }
}

/* LBM only (walkers frozen): used to spin up a flow before walkers are released */
ORC_API void orc_step_fluid(void* h, long long nsteps)
{
    orc_t* o = (orc_t*)h;
    for (long long s = 0; s < nsteps; ++s) {
        if (!o->coupling) rasterize(o, o->t);
        lbm_step(o, o->t);
        if (o->dem) dem_advance(o);
        o->t++;
    }
}

ORC_API long long orc_time(void* h) { return ((orc_t*)h)->t; }
ORC_API void orc_set_time(void* h, long long t) { ((orc_t*)h)->t = t; ((orc_t*)h)->solid_time = -1; }

ORC_API void orc_velocity(void* h, double* out)
{
    orc_t* o = (orc_t*)h;
    memcpy(out, o->u, sizeof(double) * 3 * (size_t)o->ncell);
}
ORC_API void orc_density(void* h, double* out)
{
    orc_t* o = (orc_t*)h;
    memcpy(out, o->rho, sizeof(double) * (size_t)o->ncell);
}
/* Post-collision populations f+(t-1) held at the start of step t, direction-major */
ORC_API void orc_populations(void* h, double* out)
{
    orc_t* o = (orc_t*)h;
    memcpy(out, o->f, sizeof(double) * (size_t)o->q * o->ncell);
}
ORC_API void orc_set_populations(void* h, const double* f)
{
    orc_t* o = (orc_t*)h;
    memcpy(o->f, f, sizeof(double) * (size_t)o->q * o->ncell);
}
ORC_API void orc_set_velocity(void* h, const double* u)
{
    orc_t* o = (orc_t*)h;
    memcpy(o->u, u, sizeof(double) * 3 * (size_t)o->ncell);
}
ORC_API void orc_solid(void* h, long long t, int* count, int* owner)
{
    orc_t* o = (orc_t*)h;
    if (o->solid_time != t) rasterize(o, t);
    memcpy(count, o->cnt, sizeof(int) * (size_t)o->ncell);
    memcpy(owner, o->own, sizeof(int) * (size_t)o->ncell);
}
/* Solid fraction at step t of the n listed cells only (the rule of orc_solid, cell by cell); the
 * context's own solid arrays are left as they are. */
ORC_API void orc_solid_cells(void* h, long long t, long long n, const int64_t* cells, int* count,
                             int* owner)
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    int* cand = (int*)malloc(sizeof(int) * (size_t)(o->P + 1));
    int* npart = (int*)calloc((size_t)o->P + 1, sizeof(int));
    for (long long m = 0; m < n; ++m) {
        long long c = cells[m];
        long long i = c % o->n[0], j = (c / o->n[0]) % o->n[1], k = c / ((long long)o->n[0] * o->n[1]);
        raster_cell(o, &fr, i, j, k, cand, npart, &count[m], &owner[m]);
    }
    free(cand);
    free(npart);
    frame_free(&fr);
}
ORC_API void orc_walkers(void* h, double* x, double* x0)
{
    orc_t* o = (orc_t*)h;
    memcpy(x, o->x, sizeof(double) * 3 * (size_t)o->nw);
    if (x0) memcpy(x0, o->x0, sizeof(double) * 3 * (size_t)o->nw);
}

/* Eq. 16 with m_s = 1 and dx = 1: the count of walkers per cell (Reading: the solid fraction
 * named beside Eq. 16 is reported separately, not folded in). */
ORC_API void orc_concentration(void* h, uint32_t* out)
{
    orc_t* o = (orc_t*)h;
    memset(out, 0, sizeof(uint32_t) * (size_t)o->ncell);
    for (long long w = 0; w < o->nw; ++w) out[walker_cell(o, o->x + 3 * w)]++;
}

/* Binning of caller-given binary32 positions (the exactness check of the cell assignment) */
ORC_API void orc_bin_positions(void* h, long long n, const float* pos, int64_t* cell)
{
    orc_t* o = (orc_t*)h;
    for (long long w = 0; w < n; ++w) {
        double x[3] = {pos[3 * w], pos[3 * w + 1], pos[3 * w + 2]};
        cell[w] = walker_cell(o, x);
    }
}

/* Walker moments: out = {N, mean(x - x0)[3], var(x - x0)[3], mean(x)[3], var(x)[3]}
 * (population variances, two passes). Section 4 fits the z-variance against time (Eq. 38). */
ORC_API void orc_moments(void* h, double out[13])
{
    orc_t* o = (orc_t*)h;
    for (int m = 0; m < 13; ++m) out[m] = 0.0;
    out[0] = (double)o->nw;
    if (o->nw == 0) return;
    double md[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
    for (long long w = 0; w < o->nw; ++w)
        for (int a = 0; a < 3; ++a) {
            md[a] += o->x[3 * w + a] - o->x0[3 * w + a];
            mx[a] += o->x[3 * w + a];
        }
    for (int a = 0; a < 3; ++a) { md[a] /= (double)o->nw; mx[a] /= (double)o->nw; }
    double vd[3] = {0, 0, 0}, vx[3] = {0, 0, 0};
    for (long long w = 0; w < o->nw; ++w)
        for (int a = 0; a < 3; ++a) {
            double d = o->x[3 * w + a] - o->x0[3 * w + a] - md[a];
            double e = o->x[3 * w + a] - mx[a];
            vd[a] += d * d;
            vx[a] += e * e;
        }
    for (int a = 0; a < 3; ++a) {
        out[1 + a] = md[a];
        out[4 + a] = vd[a] / (double)o->nw;
        out[7 + a] = mx[a];
        out[10 + a] = vx[a] / (double)o->nw;
    }
}

/* {sum rho, sum_i f_i e_i (3)} over all cells at the last LBM step (pre-collision) */
ORC_API void orc_mass_momentum(void* h, double out[4])
{
    orc_t* o = (orc_t*)h;
    out[0] = o->mass;
    for (int a = 0; a < 3; ++a) out[1 + a] = o->mom[a];
}

/* {F_p (3), T_p (3)} per particle at the last LBM step */
ORC_API void orc_forces(void* h, double* out)
{
    orc_t* o = (orc_t*)h;
    for (int p = 0; p < o->P; ++p)
        for (int a = 0; a < 3; ++a) {
            out[6 * p + a] = o->Fp[3 * p + a];
            out[6 * p + 3 + a] = o->Tp[3 * p + a];
        }
}

/* {type I, II, III, IV counts, bisection failures, refill failures, wall failures, seed failures} */
ORC_API void orc_counters(void* h, long long out[8])
{
    orc_t* o = (orc_t*)h;
    for (int m = 0; m < 4; ++m) out[m] = o->cnt_type[m];
    out[4] = o->bisect_fail; out[5] = o->refill_fail; out[6] = o->wall_fail; out[7] = o->seed_fail;
}

/* Sampled checks at full size: the step-t update of chosen cells from the populations now
 * held (f+(t-1)), without changing the state. fout [q n] direction-major, uout [3 n]. */
ORC_API void orc_lbm_cells(void* h, long long n, const int64_t* cells, double* fout, double* uout,
                           double* rhoout)
{
    orc_t* o = (orc_t*)h;
    if (o->solid_time != o->t) rasterize(o, o->t);
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, o->t, &fr);
    double F[3];
    body_force(o, o->t, F);
    for (long long m = 0; m < n; ++m) {
        long long c = cells[m];
        long long i = c % o->n[0], j = (c / o->n[0]) % o->n[1], k = c / ((long long)o->n[0] * o->n[1]);
        double fi[19], fo[19], u[3], rho, dp[3];
        pull_cell(o, i, j, k, fi);
        collide_cell(o, &fr, o->t, i, j, k, o->cnt[c], o->own[c], fi, F, fo, u, &rho, dp);
        for (int d = 0; d < o->q; ++d) fout[(size_t)d * n + m] = fo[d];
        for (int a = 0; a < 3; ++a) uout[3 * m + a] = u[a];
        if (rhoout) rhoout[m] = rho;
    }
    frame_free(&fr);
}

/* Sampled walker checks: advance caller-given walkers (positions x [3n], ids) by one step at
 * the current time t with the velocity field now held (set with orc_set_velocity). */
ORC_API void orc_walkers_advance(void* h, long long n, const double* x, const uint32_t* ids, double* xout)
{
    orc_t* o = (orc_t*)h;
    frame_t fr1;
    frame_alloc(o, &fr1);
    frame_at(o, o->t + 1, &fr1);
    for (long long w = 0; w < n; ++w) walker_advance(o, &fr1, o->u, ids[w], (uint32_t)o->t, x + 3 * w, xout + 3 * w);
    frame_free(&fr1);
}

/* Particle-fluid coupling: 0 partially saturated cells (default), 1 IBB (Section 2.4.3) */
ORC_API void orc_set_coupling(void* h, int mode) { ((orc_t*)h)->coupling = mode; }

ORC_API void orc_nodes(void* h, long long t, int* node) { classify_nodes((orc_t*)h, t, node); }

ORC_API double orc_ibb_q(void* h, long long t, int p, long long i, long long j, long long k, const int e[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    double qv = (double)ibb_q(o, &fr, p, i, j, k, e);
    frame_free(&fr);
    return qv;
}

ORC_API double orc_ibb_link(int q, int i, double qf, double rho_f, const double uf[3], const double uff[3],
                            const double uw[3], double Gp)
{
    return ibb_link(q, i, opposite(i), qf, rho_f, uf, uff, uw, Gp);
}

/* ---- single-function entry points for the CPU pins ---- */
ORC_API void orc_philox(uint64_t seed, const uint32_t ctr[4], uint32_t out[4])
{
    philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, out);
}

/* The three step normals of walker id at step t (counter (id, t, 0, 0)) */
ORC_API void orc_step_normals(uint64_t seed, uint32_t id, uint32_t t, double z[3])
{
    uint32_t ctr[4] = {id, t, 0u, 0u}, r[4];
    philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, r);
    box_muller(u24(r[0]), u24(r[1]), &z[0], &z[1]);
    box_muller(u24(r[2]), u24(r[3]), &z[2], NULL);
}

/* Test helper (no part of the method): the first seed in [seed0, seed0 + count) whose Philox
 * output for counter ctr has (word `word`) >> 8 == target, or -1. Tests use it to find the rare
 * counters that put a uniform at the end of its range. */
ORC_API long long orc_philox_find_seed(uint64_t seed0, long long count, const uint32_t ctr[4], int word,
                                       uint32_t target)
{
    for (long long s = 0; s < count; ++s) {
        uint32_t r[4];
        uint64_t seed = seed0 + (uint64_t)s;
        philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, r);
        if ((r[word & 3] >> 8) == target) return (long long)seed;
    }
    return -1;
}

ORC_API double orc_metaball(void* h, long long t, int p, const double x[3], double g[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    double f = f_at(o, &fr, p, x, g);
    frame_free(&fr);
    return f;
}

ORC_API float orc_metaball32(void* h, long long t, int p, const float x[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    float f = metaball32(o, &fr, p, x);
    frame_free(&fr);
    return f;
}

ORC_API double orc_bound_radius(void* h, int p) { return ((orc_t*)h)->Rb[p]; }

ORC_API int orc_inside(void* h, long long t, const double x[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    int p = inside_any64(o, &fr, x);
    frame_free(&fr);
    return p;
}

ORC_API int orc_bisect(void* h, long long t, int p, const double a[3], const double b[3], double xi[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    int ok = bisect(o, &fr, p, a, b, xi, NULL);
    frame_free(&fr);
    return ok;
}

ORC_API void orc_reflect(void* h, long long t, int p, const double xint[3], const double xf[3], double xnew[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t, &fr);
    reflect(o, &fr, p, xint, xf, xnew);
    frame_free(&fr);
}

ORC_API int orc_refill(void* h, long long t, int p, const double x[3], uint32_t id, double xnew[3])
{
    orc_t* o = (orc_t*)h;
    frame_t fr;
    frame_alloc(o, &fr);
    frame_at(o, t + 1, &fr);
    int ok = refill(o, &fr, p, x, id, (uint32_t)t, xnew);
    frame_free(&fr);
    return ok;
}

ORC_API void orc_trilinear(void* h, const double x[3], double u[3]) { trilinear((orc_t*)h, ((orc_t*)h)->u, x, u); }

ORC_API void orc_pose(void* h, long long t, int p, double org[3], double vel[3])
{
    double R[3][3];
    particle_pose((orc_t*)h, t, p, org, vel, R);
}

ORC_API void orc_lattice(int q, int* e, double* w)
{
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = lattice_e(q, i)[a];
        w[i] = lattice_weight(q, i);
    }
}

/* R_c = max_i (|c_i| + sqrt(k_i)) over particle p's body-frame control points */
static double dem_reach(const orc_t* o, int p)
{
    double r = 0.0;
    for (int i = o->coff[p]; i < o->coff[p + 1]; ++i) {
        double c = sqrt(o->cbody[3 * i] * o->cbody[3 * i] + o->cbody[3 * i + 1] * o->cbody[3 * i + 1]
                        + o->cbody[3 * i + 2] * o->cbody[3 * i + 2]);
        double e = c + sqrt(o->kc[i]);
        if (e > r) r = e;
    }
    return r;
}

/* Mass properties of particle p from its metaball (Eq. 3) at density rho: the body-frame sample
 * points (i + 1/2) h, h = 1/4, out to the bound radius, inside when the binary32 sum (the
 * operation order of metaball32, no wrapping) reaches 1. The sums of the inside points' counts,
 * coordinates and coordinate products are integers (in units of h/2), so they are exact; then
 * m = rho n h^3, the centre of mass, and the inertia tensor about it (xx yy zz xy xz yz). */
#define DEM_MASS_H 0.25
static void dem_mass(const orc_t* o, int p, double rho, double out[10])
{
    int N = (int)ceil(o->Rb[p] / DEM_MASS_H) + 1;
    long long n = 0, S1[3] = {0, 0, 0}, S2[6] = {0, 0, 0, 0, 0, 0};
    for (int k = -N; k < N; ++k)
        for (int j = -N; j < N; ++j)
            for (int i = -N; i < N; ++i) {
                int a = 2 * i + 1, b = 2 * j + 1, c = 2 * k + 1;
                float x[3] = {(float)a * 0.125f, (float)b * 0.125f, (float)c * 0.125f};
                float f = 0.0f;
                for (int m = o->coff[p]; m < o->coff[p + 1]; ++m) {
                    float dx = x[0] - (float)o->cbody[3 * m];
                    float dy = x[1] - (float)o->cbody[3 * m + 1];
                    float dz = x[2] - (float)o->cbody[3 * m + 2];
                    float xx = dx * dx;
                    float yy = dy * dy;
                    float zz = dz * dz;
                    float r2 = xx + yy;
                    r2 = r2 + zz;
                    f = f + o->kc32[m] / r2;
                }
                if (f >= 1.0f) {
                    n++;
                    S1[0] += a; S1[1] += b; S1[2] += c;
                    S2[0] += (long long)a * a; S2[1] += (long long)b * b; S2[2] += (long long)c * c;
                    S2[3] += (long long)a * b; S2[4] += (long long)a * c; S2[5] += (long long)b * c;
                }
            }
    double dn = (double)n;
    out[0] = rho * (dn * 0.015625);
    double cm[3];
    for (int e = 0; e < 3; ++e) { cm[e] = ((double)S1[e] * 0.125) / dn; out[1 + e] = cm[e]; }
    static const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    double J[6], w = rho * 0.015625;
    for (int m = 0; m < 6; ++m) J[m] = ((double)S2[m] * 0.015625 - (dn * cm[ia[m]]) * cm[ib[m]]) * w;
    out[4] = J[1] + J[2];
    out[5] = J[0] + J[2];
    out[6] = J[0] + J[1];
    out[7] = -J[3];
    out[8] = -J[4];
    out[9] = -J[5];
}

/* Free DEM set-up: contact law, gravity, DEM steps per LBM step, hydrodynamic coupling on/off,
 * and per particle the density, sphere radius R_s, initial velocity and spin (NULL: those of the
 * prescribed motion at the current time). Mass, centre of mass and inertia follow from the
 * metaball (dem_mass); the body frame is then moved to the centre of mass (control points
 * c_i - c_m rounded to binary32, origin + c_m), so that the state's origin is the centre of
 * mass and the fluid's torque is taken about it. The state starts at the prescribed origin of
 * the current time with the body frame as given (identity orientation). Returns 0, or -1 for
 * an invalid set-up. */
ORC_API int orc_set_dem(void* h, double kn, double etan, double kt, double etat, double mus,
                        const double g[3], int nsub, int hydro, const double* density,
                        const double* Rs, const double* v0, const double* w0)
{
    orc_t* o = (orc_t*)h;
    int P = o->P;
    if (nsub < 1 || P < 1 || kn < 0.0 || etan < 0.0 || kt < 0.0 || etat < 0.0 || mus < 0.0)
        return -1;
    for (int p = 0; p < P; ++p)
        if (!(density[p] > 0.0) || !(Rs[p] > 0.0)) return -1;
    double* mp = (double*)malloc(sizeof(double) * 10 * (size_t)P);
    for (int p = 0; p < P; ++p) {
        dem_mass(o, p, density[p], mp + 10 * p);
        if (!(mp[10 * p] > 0.0)) { free(mp); return -1; }
    }
    /* recentre the body frames on the centres of mass */
    for (int p = 0; p < P; ++p) {
        const double* cm = mp + 10 * p + 1;
        for (int i = o->coff[p]; i < o->coff[p + 1]; ++i)
            for (int a = 0; a < 3; ++a) o->cbody[3 * i + a] = (double)(float)(o->cbody[3 * i + a] - cm[a]);
        o->Rb[p] = bound_radius(o, p);
        if (!(Rs[p] < dem_reach(o, p))) { free(mp); return -1; }
    }
    free(o->dst); free(o->dmass); free(o->dIb); free(o->dRs); free(o->dzoom); free(o->dcm);
    free(o->dxi); free(o->dxm); free(o->dact); free(o->dxiw); free(o->dxmw); free(o->dactw);
    size_t PP = (size_t)P * P;
    o->dst = (double*)calloc(13 * (size_t)P, sizeof(double));
    o->dmass = (double*)malloc(sizeof(double) * (size_t)P);
    o->dIb = (double*)malloc(sizeof(double) * 6 * (size_t)P);
    o->dRs = (double*)malloc(sizeof(double) * (size_t)P);
    o->dzoom = (double*)malloc(sizeof(double) * (size_t)P);
    o->dcm = mp;
    o->dxi = (double*)calloc(3 * PP, sizeof(double));
    o->dxm = (double*)calloc(3 * PP, sizeof(double));
    o->dact = (unsigned char*)calloc(PP, 1);
    o->dxiw = (double*)calloc(18 * (size_t)P, sizeof(double));
    o->dxmw = (double*)calloc(18 * (size_t)P, sizeof(double));
    o->dactw = (unsigned char*)calloc(6 * (size_t)P, 1);
    o->dem_kn = kn; o->dem_etan = etan; o->dem_kt = kt; o->dem_etat = etat; o->dem_mus = mus;
    for (int a = 0; a < 3; ++a) o->dem_g[a] = g[a];
    o->dem_nsub = nsub;
    o->dem_hydro = hydro ? 1 : 0;
    for (int p = 0; p < P; ++p) {
        double org[3], vel[3], R[3][3];
        particle_pose(o, o->t, p, org, vel, R);
        double* st = o->dst + 13 * (size_t)p;
        for (int a = 0; a < 3; ++a) {
            st[a] = org[a] + mp[10 * p + 1 + a];
            st[7 + a] = v0 ? v0[3 * p + a] : vel[a];
            st[10 + a] = w0 ? w0[3 * p + a] : o->omg[3 * p + a];
        }
        st[3] = 1.0; st[4] = st[5] = st[6] = 0.0;
        o->dmass[p] = mp[10 * p];
        for (int m = 0; m < 6; ++m) o->dIb[6 * p + m] = mp[10 * p + 4 + m];
        o->dRs[p] = Rs[p];
        o->dzoom[p] = 1.0 - Rs[p] / dem_reach(o, p);
    }
    o->dem = 1;
    o->dem_nodes_t = -2;
    o->solid_time = -1;
    return 0;
}

/* Mass properties of the free-DEM particles: out[10 p ..] = mass, centre of mass in the original
 * body frame (3), inertia about it (xx yy zz xy xz yz) */
ORC_API void orc_dem_mass(void* h, double* out)
{
    orc_t* o = (orc_t*)h;
    if (o->dem) memcpy(out, o->dcm, sizeof(double) * 10 * (size_t)o->P);
}

ORC_API void orc_particle_state(void* h, double* out)
{
    orc_t* o = (orc_t*)h;
    if (o->dem) memcpy(out, o->dst, sizeof(double) * 13 * (size_t)o->P);
}

ORC_API void orc_set_particle_state(void* h, const double* st)
{
    orc_t* o = (orc_t*)h;
    if (o->dem) memcpy(o->dst, st, sizeof(double) * 13 * (size_t)o->P);
    o->solid_time = -1;
}

/* Contact geometry of pair (i, j) in the current state, as a new contact (Eqs. 7-9):
 * out = x_m[3], x_c0[3], x_c1[3], n[3], delta, x_cp[3] */
ORC_API void orc_dem_pair_geom(void* h, int i, int j, double* out)
{
    orc_t* o = (orc_t*)h;
    double* cbuf = (double*)malloc(sizeof(double) * (6 * (size_t)o->Nc + 6));
    double* kbuf = (double*)malloc(sizeof(double) * (2 * (size_t)o->Nc + 2));
    const double* si = o->dst + 13 * (size_t)i;
    double oj[3];
    dem_image(o, si, o->dst + 13 * (size_t)j, oj);
    int n0 = dem_internal(o, i, si, cbuf, kbuf);
    int n1 = dem_internal(o, j, oj, cbuf + 3 * n0, kbuf + n0);
    double xm[3];
    out[12] = dem_pair_geom(cbuf, kbuf, n0, cbuf + 3 * n0, kbuf + n0, n1, o->dRs[i], o->dRs[j], 0, xm,
                            out + 3, out + 6, out + 9, out + 13);
    for (int a = 0; a < 3; ++a) out[a] = xm[a];
    free(cbuf); free(kbuf);
}

/* Contact geometry of particle p and wall face f = 2 axis + side, as a new contact (Eqs. 10-11):
 * out = x_cm[3], x_cw[3], n[3], delta, x_cp[3] */
ORC_API void orc_dem_wall_geom(void* h, int p, int f, double* out)
{
    orc_t* o = (orc_t*)h;
    double* cbuf = (double*)malloc(sizeof(double) * (3 * (size_t)o->Nc + 3));
    double* kbuf = (double*)malloc(sizeof(double) * ((size_t)o->Nc + 1));
    int n = dem_internal(o, p, o->dst + 13 * (size_t)p, cbuf, kbuf);
    out[9] = dem_wall_geom(cbuf, kbuf, n, f >> 1, f & 1, (double)o->n[f >> 1], o->dRs[p], 0, out, out + 3,
                           out + 6, out + 10);
    free(cbuf); free(kbuf);
}

/* The contact law alone (normal spring-dashpot and Eq. 5) with the context's DEM parameters:
 * the force on body i for overlap delta, unit normal n from i towards the other body,
 * contact-point velocities vi, vj and DEM step dt. xi is the contact's tangential spring, read
 * and updated in place. */
ORC_API void orc_dem_contact_force(void* h, double delta, const double n[3], const double vi[3],
                                   const double vj[3], double dt, double xi[3], double F[3])
{
    dem_contact_force((const orc_t*)h, delta, n, vi, vj, dt, xi, F);
}

/* DEM steps alone (no fluid, no walkers): the hydrodynamic force and torque are those of the
 * last LBM update when the coupling is on */
ORC_API void orc_dem_advance(void* h, long long nsteps)
{
    orc_t* o = (orc_t*)h;
    for (long long s = 0; s < nsteps; ++s) dem_advance(o);
}

/* IBB with the free DEM: the node classes of time t_prev (0 fluid, 1 + particle), which the
 * step at t_prev + 1 refills from */
ORC_API void orc_set_prev_nodes(void* h, long long t_prev, const int* nodes)
{
    orc_t* o = (orc_t*)h;
    if (!o->dem_nodes) o->dem_nodes = (int*)malloc(sizeof(int) * (size_t)o->ncell);
    memcpy(o->dem_nodes, nodes, sizeof(int) * (size_t)o->ncell);
    o->dem_nodes_t = t_prev;
}
