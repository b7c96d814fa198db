/*
 * rwmi.h -- C ABI of the GB300 (sm_103a) fluid-solute step of RW-MI-DELBM
 * (Zhao, Zhang, Li and Galindo-Torres, arXiv 2308.05007).
 *
 * One timestep t -> t+1 of a simulation context runs, on one GPU:
 *   - the prescribed rigid motion of metaball particles (Eq. 3 shapes; the DEM of Eq. 4 is
 *     held to given trajectories) and their partially-saturated solid fraction per cell;
 *   - a fused lattice Boltzmann pull-stream + BGK collide (Eqs. 12-15; D3Q19 as in Section 2.3,
 *     or D3Q15) with partially-saturated-cell solid coupling and Guo body forcing, which also
 *     yields the hydrodynamic force and torque on every particle;
 *   - the random-walk advance of every solute walker (Eq. 2) with the velocity interpolated
 *     from the lattice (Section 2.4.1) and the walker/particle rules of Section 2.4.2:
 *     refill of type II walkers, Algorithm 1 (bisection) and Algorithm 2 (specular
 *     reflection) for type IV walkers, free motion for types I and III;
 *   - on request or at a set cadence: the counting sort of walkers by cell whose histogram is
 *     the concentration of Eq. 16, and FP64 walker moments (the input of Eqs. 38-40).
 *
 * Conventions for every entry point:
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3, kinematic viscosity (tau - 1/2)/3.
 *   - Cell (i, j, k) is [i, i+1) x [j, j+1) x [k, k+1); its lattice node sits at the centre.
 *     Flat cell index c = i + nx (j + ny k). Walker positions are unwrapped.
 *   - Ownership: the library owns all device state and allocates it in rwmi_create,
 *     rwmi_set_metaballs and rwmi_seed_walkers / rwmi_set_walkers. The caller owns every input
 *     and output array; inputs are copied during the call. An output pointer may be host
 *     (pageable or pinned) or device memory of the context's GPU; the library tells them apart
 *     with cudaPointerGetAttributes.
 *   - Streams: all GPU work of a context is issued on one stream (rwmi_set_stream; default: a
 *     stream the context creates). rwmi_step is asynchronous; getters synchronise that stream.
 *     Copies and allocations are ordered on that stream too (stream-ordered allocator), so
 *     creating, reading or destroying one context never waits for another context's work.
 *     A device array the caller passes must be ready before the call (its producer finished or
 *     ordered before the context's stream).
 *   - Errors: every call returns an rwmi_status. RWMI_E_INVALID and RWMI_E_STATE (a call made
 *     in the wrong state) leave the context unchanged. RWMI_E_NONFINITE reports non-finite
 *     values in the state; the context still answers, so the state can be read out.
 *     RWMI_E_OOM and RWMI_E_CUDA fence the context: its device state may be half built, so
 *     every later call on it except rwmi_last_error, rwmi_launch_count and rwmi_destroy
 *     returns RWMI_E_STATE, and rwmi_last_error keeps the message of the failure that fenced
 *     it. Positive values are warnings. Nothing is thrown across the ABI; nothing exits.
 *     Calls on one context are not thread-safe.
 */
#ifndef RWMI_H
#define RWMI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define RWMI_API __attribute__((visibility("default")))
#else
#define RWMI_API
#endif

typedef struct rwmi_ctx rwmi_ctx;

typedef enum {
    RWMI_OK = 0,
    RWMI_W_BISECT = 1,       /* Algorithm 1 found no point with |f - 1| < 1e-3 in 200 steps for
                                some walker (Section 2.4.2: "an error is reported"); the walker
                                stayed where it was. Also refill failures. */
    RWMI_W_SEED = 2,         /* some walker found no free seed point (see rwmi_seed_walkers) */
    RWMI_BUSY = 3,           /* rwmi_query: GPU work of the context is still running */
    RWMI_E_INVALID = -1,     /* bad argument or size; context unchanged */
    RWMI_E_OOM = -2,         /* a device (or host) allocation failed; fences the context */
    RWMI_E_CUDA = -3,        /* a CUDA runtime call or kernel launch failed; fences the context */
    RWMI_E_NONFINITE = -4,   /* NaN/Inf in the FP64 mass sum or a walker velocity */
    RWMI_E_TIMEOUT = -5,     /* a bounded device wait gave up */
    RWMI_E_STATE = -6        /* call out of order (e.g. configuring after the first step), or
                                any call on a context fenced by RWMI_E_OOM / RWMI_E_CUDA */
} rwmi_status;

/* Storage of the populations in HBM and the arithmetic of the LBM update. The walkers, the
 * rasteriser and the velocity field handed to the walkers are binary32 in every case. */
enum {
    RWMI_STORE_FP32 = 0,          /* f_i as binary32, binary32 arithmetic */
    RWMI_STORE_FP32_SHIFT = 1,    /* f_i - w_i rho0 as binary32, binary32 arithmetic (default;
                                     keeps u ~ 1e-4 exact to ~1e-7 relative) */
    RWMI_STORE_FP16_SHIFT = 2,    /* f_i - w_i rho0 as binary16, binary32 arithmetic */
    RWMI_STORE_FP64_SHIFT = 3     /* f_i - w_i rho0 as binary64, binary64 arithmetic: the
                                     FP64-on-GPU reference run (GB300's FP64 rate is low) */
};

typedef struct {
    int32_t q;                 /* 15 (D3Q15) or 19 (D3Q19, Section 2.3). Default 19. */
    int32_t storage;           /* RWMI_STORE_*. Default RWMI_STORE_FP32_SHIFT. */
    uint32_t wall_mask;        /* bit a: no-slip walls on both faces normal to axis a
                                  (half-way bounce-back for the fluid, specular reflection for
                                  walkers). Other axes are periodic. Default 0. */
    double body_force[3];      /* force density F0 (lattice units). Default 0. */
    double force_period;       /* F(t) = F0 sin(2 pi t / force_period); 0: constant F0 */
    double rho0;               /* reference density (initial state, shift). Default 1. */
    double init_velocity[3];   /* initial equilibrium velocity. Default 0. */
    int32_t sort_interval;     /* sort walkers by cell every this many steps (0: never).
                                  Default 16. The sort also refreshes the concentration. */
    int32_t moment_interval;   /* append FP64 walker moments to the series every this many
                                  steps (0: never). Default 0. */
    int32_t use_graphs;        /* replay captured CUDA graphs for repeated steps. Default 1. */
    int32_t lbm_block;         /* threads per block of the LBM kernel: 64, 128 or 256 (0: 256).
                                  Default 128 (in the overlapped step the smaller blocks share
                                  the SMs with the raster better); rwmi_autotune picks it by
                                  timing the update alone. */
    int32_t overlap;           /* step schedule, same results bit for bit in every case:
                                  0: one stream, phases one after the other;
                                  1: the raster of t+1 on a second stream while the LBM of t runs
                                     (ALU-bound beside HBM-bound);
                                  2: as 1, and the walkers of t (with sort and moments) on a third
                                     stream beside the fluid of t+1. Default 2. */
    int32_t coupling;          /* particle-fluid coupling of the LBM: 0 partially saturated cells
                                  (Noble-Torczynski; default); 1 the paper's own (Section 2.4.3):
                                  interpolated bounce-back on the moving metaball surface
                                  (Eqs. 23-25), Galilean-invariant momentum exchange for the
                                  force, refilling of uncovered nodes (Eq. 27). IBB requires
                                  storage FP32_SHIFT or FP64_SHIFT (else RWMI_E_INVALID). */
    int32_t lbm_staging;       /* 1: the LBM update (partially saturated cells, binary32 or
                                  binary16 storage, nx a multiple of 4 (binary32) or 8 (binary16))
                                  stages its pulled rows through shared memory with TMA tensor
                                  copies; 0: direct coalesced loads. Same results bit for bit.
                                  Default 0 (direct loads measured faster on GB300); ignored where
                                  not supported. */
    int32_t force_interval;    /* record every particle's force and torque every this many steps
                                  (0: never; rwmi_force_series reads them). A recorded step runs
                                  the fused update-and-reduce LBM pass (binary16 and plain
                                  binary32 storage: the update and a reduce-only pass), whose
                                  stored populations equal the plain update's, so the trajectory
                                  does not depend on the interval. Default 0. */
} rwmi_config;

/* Fills *cfg with the defaults listed above. */
RWMI_API void rwmi_config_defaults(rwmi_config* cfg);

/* Creates a context for a box of dims[0] x dims[1] x dims[2] cells on the current CUDA
 * device, with BGK relaxation time tau (Eq. 12; tau > 1/2), walker diffusion coefficient D
 * (Eq. 2; D >= 0) and the 64-bit Philox key seed that fixes all walker noise. The context
 * takes the default configuration; change it with rwmi_configure before the first step.
 * Sizes: each dim >= 1; total cells <= 2^31 - 1. */
RWMI_API rwmi_status rwmi_create(rwmi_ctx** ctx, const int32_t dims[3], double tau, double D,
                                 uint64_t seed);

/* Replaces the configuration. Allowed only before the first rwmi_step; resets the fluid to
 * the equilibrium at (rho0, init_velocity). */
RWMI_API rwmi_status rwmi_configure(rwmi_ctx* ctx, const rwmi_config* cfg);

/* Issues all later GPU work of the context on this cudaStream_t (e.g. a torch stream). */
RWMI_API rwmi_status rwmi_set_stream(rwmi_ctx* ctx, void* cuda_stream);

/* Metaball particles, Eq. 3: particle p owns control points center_offsets[p] ..
 * center_offsets[p+1]-1, with body-frame positions centers_body[3 i .. 3 i + 2] relative to
 * the particle origin and weights k[i] > 0 (f(x) = sum k_i / |x - x_i|^2, inside where f >= 1).
 * The origin follows origin + amplitude sin(2 pi t / period + phase) (period 0: at rest) and
 * the body spins with constant angular velocity omega (rad per step, may be NULL for none).
 * Arrays: center_offsets [P+1], centers_body [3 Nc], k [Nc], origin/amplitude/omega [3P],
 * period/phase [P], host memory. Limits: P <= 511, Nc <= 65535. Replaces earlier particles.
 * Allowed before the first step only. */
RWMI_API rwmi_status rwmi_set_metaballs(rwmi_ctx* ctx, int32_t n_particles,
                                        const int32_t* center_offsets, const float* centers_body,
                                        const float* k, const double* origin,
                                        const double* amplitude, const double* period,
                                        const double* phase, const double* omega);

/* ---- Free DEM (Section 2.2, Eqs. 4-11) ------------------------------------------------------
 * Instead of their prescribed trajectories the particles can move freely: Eq. 4 (Newton's and
 * Euler's equations) under gravity, contact forces and the fluid's force and torque. Contacts
 * use the sphero-metaball of Eqs. 6-11: the metaball scaled about its body origin by
 * s = 1 - R_s / R_c (R_c = max_i |c_i| + sqrt(k_i)) and dilated by the sphere radius R_s; pair
 * geometry by Newton-Raphson on grad(f_0 + f_1) = 0 (Eq. 7) and Eq. 8 solved for f = 1 along the
 * gradient; wall geometry (faces of walled axes) by Newton-Raphson for the point of the scaled
 * surface closest to the face. Normal force: linear spring-dashpot, k_n delta plus eta_n times
 * the approach speed, never attractive. Tangential force: Eq. 5, a spring k_t xi plus damping
 * eta_t, limited to mu_s times the normal force. Integration per DEM step dt = 1 / substeps:
 * symplectic Euler for the origin, explicit Euler for the spin (world frame, gyroscopic term
 * included) and a normalised first-order quaternion update for the orientation. The fluid force
 * and torque of step t's LBM update act over its DEM steps (hydro = 1). The arithmetic is
 * binary64 without contraction, so with hydro = 0 trajectories equal the CPU oracle's. */
typedef struct {
  double kn, eta_n;       /* normal stiffness and damping (lattice units) */
  double kt, eta_t;       /* tangential stiffness and damping (Eq. 5) */
  double mu_s;            /* static friction coefficient (Eq. 5) */
  double gravity[3];      /* g of Eq. 4 */
  int32_t substeps;       /* DEM steps per LBM step, >= 1 */
  int32_t hydro;          /* 1: F^e, T^e of Eq. 4 are the fluid's force and torque; 0: none */
} rwmi_dem_config;

/* kn 200, eta_n 0, kt 0, eta_t 0, mu_s 0, gravity 0, substeps 10, hydro 1 */
RWMI_API void rwmi_dem_defaults(rwmi_dem_config* cfg);

/* Switches the current particles to the free DEM from the current time. Per particle (host
 * arrays): density [P] > 0, sphere radius R_s [P], initial velocity and spin [3 P] (NULL: those
 * of the prescribed motion at the current time). Mass, centre of mass and inertia tensor come
 * from the metaball itself: body-frame sample points (i + 1/2) h, h = 1/4, inside when the
 * binary32 sum of Eq. 3 reaches 1, summed exactly as integers (rwmi_particle_mass). The body
 * frame is then moved to the centre of mass (control points c_i - c_m in binary32), so the
 * state's origin is the centre of mass. The state starts at the prescribed origin of the
 * current time (plus c_m) with the body frame as given. Requires 0 < R_s < max |c_i - c_m| +
 * sqrt(k_i), binary32-shifted or binary64 storage, and at most 16 control points per particle;
 * either coupling (with IBB the node classes of t - 1 are those of the previous step, and at the
 * first step of the free run those of t). Every step then forms the fluid force in the LBM
 * update itself (one fused pass). RWMI_E_INVALID otherwise (context unchanged), RWMI_E_STATE if
 * the particles are free already. Before the first step. */
RWMI_API rwmi_status rwmi_set_dem(rwmi_ctx* ctx, const rwmi_dem_config* cfg, const double* density,
                                  const double* sphere_radius, const double* velocity,
                                  const double* spin);

/* Mass properties of the free particles, out[10 p .. 10 p + 9] = mass, centre of mass in the body
 * frame given to rwmi_set_metaballs (3), inertia tensor about it (xx, yy, zz, xy, xz, yz). */
RWMI_API rwmi_status rwmi_particle_mass(rwmi_ctx* ctx, double* out);

/* Free-DEM state, out[13 p .. 13 p + 12] = origin (unwrapped) x y z, orientation quaternion
 * w x y z, velocity, spin (world frame), binary64; RWMI_E_STATE without rwmi_set_dem. */
RWMI_API rwmi_status rwmi_particle_state(rwmi_ctx* ctx, double* out);

/* Overwrites the free-DEM state (same layout, host array) and rebuilds the particle frame of
 * the current time; contact memory (springs) is kept. */
RWMI_API rwmi_status rwmi_set_particle_state(rwmi_ctx* ctx, const double* state);

/* Seeds n walkers uniformly in the fluid part of the box [box_lo, box_hi] (inside the domain)
 * at the current time. Walker w draws Philox counters (w, a, 2, 0), a = 0, 1, ..., < 1000,
 * takes the point box_lo + U (box_hi - box_lo) and keeps the first one outside every particle
 * (Section 2.4.2 removes walkers that start inside; drawing again keeps the count exact).
 * Returns RWMI_W_SEED if some walker found no free point (it is then left at its last draw).
 * Walker ids are 0 .. n-1; start positions are kept for rwmi_walker_moments. n <= 2^31 - 1. */
RWMI_API rwmi_status rwmi_seed_walkers(rwmi_ctx* ctx, int64_t n, const double box_lo[3],
                                       const double box_hi[3]);

/* Sets n walkers at the given binary32 positions pos[3 w .. 3 w + 2] (host or device), with
 * ids 0 .. n-1 and start positions equal to pos. Positions on walled axes must lie in [0, n]. */
RWMI_API rwmi_status rwmi_set_walkers(rwmi_ctx* ctx, int64_t n, const float* pos);

/* Advances n timesteps (asynchronous on the context's stream). Step t: solid fraction from
 * the particles at t, LBM at t, walkers from t to t+1 with the particles at t+1; walker noise
 * uses Philox counter (walker id, t, 0, 0). n >= 0. */
RWMI_API rwmi_status rwmi_step(rwmi_ctx* ctx, int32_t n);

/* Phases of one timestep, for rwmi_step_timed. */
enum {
    RWMI_PHASE_RASTER = 0,   /* solid fraction of the particles at t */
    RWMI_PHASE_LBM = 1,      /* fused pull-stream + collide at t */
    RWMI_PHASE_POSE = 2,     /* particle poses, brick lists and body force of t+1 */
    RWMI_PHASE_WALKERS = 3,  /* walker advance t -> t+1 */
    RWMI_PHASE_SORT = 4,     /* counting sort / binning (every sort_interval steps) */
    RWMI_PHASE_MOMENTS = 5,  /* moment series (every moment_interval steps) */
    RWMI_NPHASE = 6
};

/* Like rwmi_step but launches each step without graphs and brackets every phase with CUDA
 * events on the context's stream; waits for completion and adds the GPU time of each phase
 * (milliseconds, summed over the n steps) to phase_ms[RWMI_NPHASE]. Same results as rwmi_step. */
RWMI_API rwmi_status rwmi_step_timed(rwmi_ctx* ctx, int32_t n, double* phase_ms);

/* Times the LBM kernel on the current state for each block size (64, 128, 256), writing only the
 * idle population buffer and the velocity field (both are overwritten by the next step), and
 * keeps the fastest in the configuration; *chosen (may be NULL) receives it. A project-written
 * tuner: small or oddly shaped boxes favour smaller blocks. */
RWMI_API rwmi_status rwmi_autotune(rwmi_ctx* ctx, int32_t* chosen);

/* Non-blocking: RWMI_BUSY while GPU work of the context is in flight, RWMI_OK when it is idle. */
RWMI_API rwmi_status rwmi_query(rwmi_ctx* ctx);

/* Device memory a context of these sizes needs, in bytes (populations, velocity, solid words,
 * bricks, walkers with their sort and resolve buffers, particle tables), before it is created;
 * used to admit work by HBM footprint. */
RWMI_API rwmi_status rwmi_footprint(const int32_t dims[3], int32_t q, int32_t storage, int64_t n_walkers,
                                    int32_t n_particles, int32_t n_centers, uint64_t* bytes);

/* Waits for the context's stream and returns the first pending device condition:
 * RWMI_E_NONFINITE, RWMI_W_BISECT, or RWMI_OK. Clears the warning counters it reports. */
RWMI_API rwmi_status rwmi_sync(rwmi_ctx* ctx);

/* Number of completed steps. */
RWMI_API rwmi_status rwmi_time(rwmi_ctx* ctx, int64_t* t);

/* Sizes of the context: out = {nx, ny, nz, q, storage, walkers, particles, completed steps}. */
RWMI_API rwmi_status rwmi_info(rwmi_ctx* ctx, int64_t out[8]);

/* Eq. 16 with m_s = 1, dx = 1: out[c] = number of walkers in cell c (uint32, nx*ny*nz). */
RWMI_API rwmi_status rwmi_concentration(rwmi_ctx* ctx, uint32_t* out);

/* FP64 walker moments of the current positions x and start positions x0:
 * out = {N, mean(x - x0)[3], var(x - x0)[3], mean(x)[3], var(x)[3]} (population variances).
 * Section 4 fits the z-variance against time (Eq. 38) to get the dispersion coefficient. */
RWMI_API rwmi_status rwmi_walker_moments(rwmi_ctx* ctx, double out[13]);

/* The moments recorded every moment_interval steps: up to max_rows rows of
 * {t, the 13 values above}; *n_rows receives the number written (oldest first). */
RWMI_API rwmi_status rwmi_moment_series(rwmi_ctx* ctx, double* out, int32_t max_rows,
                                        int32_t* n_rows);

/* Velocity of the last LBM step, u = (sum_i f_i e_i + F/2) / rho (Eq. 15 with Guo's half
 * force): out[3 c + a], binary32, 3*nx*ny*nz values. */
RWMI_API rwmi_status rwmi_velocity(rwmi_ctx* ctx, float* out);

/* Density of the last LBM step (Eq. 14), binary32, nx*ny*nz values. */
RWMI_API rwmi_status rwmi_density(rwmi_ctx* ctx, float* out);

/* Populations now held (post-collision of the last step, f_i unshifted) as FP64:
 * out[i * ncell + c], directions in the library's order (rwmi_lattice). */
RWMI_API rwmi_status rwmi_populations(rwmi_ctx* ctx, double* out);

/* The library's velocity set: e[3 i + a] (int32) and w[i] (double) for its q directions. */
RWMI_API rwmi_status rwmi_lattice(rwmi_ctx* ctx, int32_t* e, double* w, int32_t* q);

/* Solid fraction data of the current time t (rasterised by the last step or at set-up):
 * count[c] (0..64 sub-samples inside a particle, epsilon = count / 64) and owner[c] (particle
 * index, -1 if none). With the IBB coupling the steps skip the per-cell counts (the update reads
 * node classes), so this call rasterises the current time's cells itself: one raster launch on
 * the context's stream, leaving the walkers' masks and the trajectory unchanged. */
RWMI_API rwmi_status rwmi_solid(rwmi_ctx* ctx, int32_t* count, int32_t* owner);

/* IBB node classes of the current time (Section 2.4.3, the coupling = 1 reading): out[c] = 0 for a
 * fluid node, 1 + p when the cell centre lies inside particle p (Eq. 3 >= 1 in binary32, lowest
 * index). Computed on demand with any coupling. out: int32[ncell], host or device. */
RWMI_API rwmi_status rwmi_nodes(rwmi_ctx* ctx, int32_t* out);

/* {sum rho, sum_i f_i e_i (3 components)} over all cells at the last LBM step (FP64 sums;
 * formed on the last step of every rwmi_step call). */
RWMI_API rwmi_status rwmi_mass_momentum(rwmi_ctx* ctx, double out[4]);

/* Hydrodynamic force and torque on each particle at the last LBM step, FP64:
 * out[6 p .. 6 p + 2] = F_p, out[6 p + 3 .. 6 p + 5] = T_p about the particle origin. */
RWMI_API rwmi_status rwmi_particle_forces(rwmi_ctx* ctx, double* out);

/* The forces recorded every force_interval steps (Section 2.4.3 / PSM: the force of the LBM
 * update of step t, labelled t + 1, the steps completed): the newest min(max_rows, recorded,
 * 4096) rows, oldest first, each {t + 1, F_0, T_0, F_1, T_1, ...} (1 + 6 P doubles); *n_rows is
 * set. RWMI_E_INVALID without particles or with force_interval 0. */
RWMI_API rwmi_status rwmi_force_series(rwmi_ctx* ctx, double* out, int32_t max_rows, int32_t* n_rows);

/* Walker state: out[4 w .. 4 w + 3] = {x, y, z, id} (binary32; id as a float-coded integer)
 * in the library's current (cell-sorted) order; x0 (may be NULL) receives the start
 * positions, 3 per walker, in the same order. */
RWMI_API rwmi_status rwmi_walkers(rwmi_ctx* ctx, float* out, float* x0);

/* Device counters since creation: {type I (not counted, 0), type II, III, IV walker steps,
 * Algorithm 1 failures, refill failures, wall failures, seed failures, walker steps with a
 * non-finite velocity or proposed position (that walker keeps its position), over-long walker
 * steps (resolved against all particles), walkers sent to the particle-resolution pass,
 * (cell, particle) pairs the rasteriser evaluated sub-sample by sub-sample}. */
RWMI_API rwmi_status rwmi_counters(rwmi_ctx* ctx, int64_t out[12]);

/* Checkpoint and restart: populations, walkers (positions, start positions), the step
 * counter, the particle table and, in free-DEM runs, the particle state and contact memory. A
 * restart continues bit-identically (noise is keyed by walker id and step). A free-DEM
 * checkpoint loads into a context set up with rwmi_set_dem for the same particles. */
RWMI_API rwmi_status rwmi_save(rwmi_ctx* ctx, const char* path);
RWMI_API rwmi_status rwmi_load(rwmi_ctx* ctx, const char* path);

/* ---- Batched contexts ------------------------------------------------------------------
 * Many independent simulations (each its own context: box, particles, walkers, tau, D) advanced
 * together. Each chunk of steps of every context is captured once into one CUDA graph; later
 * chunks replay it, so one graph launch advances all contexts. In the fused form (default where
 * allowed, see rwmi_batch_set_mode) each phase is one launch over all contexts' work; otherwise
 * the graph holds one concurrent branch per context. Either way the step of each context is its
 * rwmi_step (same kernel bodies, same results bit for bit). The paper has no batching; each
 * context follows the same equations as rwmi_step. */
typedef struct rwmi_batch rwmi_batch;

/* Groups n contexts (not owned: they must outlive the batch). All must share the chunk length
 * lcm(2, sort_interval, moment_interval) <= 64. Streams of the contexts should be distinct for
 * the branches to overlap. */
RWMI_API rwmi_status rwmi_batch_create(rwmi_batch** batch, rwmi_ctx* const* ctxs, int32_t n);

/* Advances every context by n steps (a multiple of the chunk; every context at a chunk
 * boundary, else RWMI_E_STATE). Asynchronous; later work on each context's stream waits for it. */
RWMI_API rwmi_status rwmi_batch_step(rwmi_batch* batch, int32_t n);

/* Waits for the batch and returns the worst rwmi_sync status of its contexts. */
RWMI_API rwmi_status rwmi_batch_sync(rwmi_batch* batch);

/* Execution form of a batch. RWMI_BATCH_FUSED runs each phase of the step (poses and bricks,
 * raster, LBM, both walker passes, the counting sort, moments) as ONE launch for all contexts:
 * every block of the launch is mapped to (context, block of the grid that context's own launch
 * would have) through a block map built at the first step, so the launch count per step no
 * longer grows with the number of contexts. It needs partially saturated cells, prescribed particles, and one velocity set,
 * storage, sort and moment interval for all contexts. Its schedule is rwmi_step's pipelined one
 * over all contexts at once: the raster of t+1 beside the LBM of t, the walkers of t beside the
 * fluid of t+1. Per-cell and per-walker results are those of rwmi_step bit for bit; the FP64
 * mass/momentum sums add binary32 block partials, so another LBM block size (see the tiles)
 * changes them at rounding level. RWMI_BATCH_BRANCHES captures the per-context steps as
 * concurrent graph branches (any configuration). RWMI_BATCH_AUTO (the default) is FUSED where
 * allowed and the contexts average under 2^19 cells (there launch gaps dominate), else
 * BRANCHES (larger domains pipeline their phases better independently). */
enum { RWMI_BATCH_AUTO = 0, RWMI_BATCH_BRANCHES = 1, RWMI_BATCH_FUSED = 2 };
/* RWMI_E_INVALID (no change) when FUSED is asked of contexts it cannot run. */
RWMI_API rwmi_status rwmi_batch_set_mode(rwmi_batch* batch, int32_t mode);

/* Work split of the fused launches (the "tiles"): threads per LBM block (64, 128, 256; one cell
 * per thread), 256-walker chunks per walker block (1..64), walkers per block of the particle-
 * resolution pass (>= 256; at most the single-context grid), bricks per raster block (>= 1).
 * Defaults {128, 1, 8192, 64}. Setting them drops the captured graphs (re-captured at the next
 * step). Results do not depend on them. */
typedef struct {
  int32_t lbm_block;
  int32_t walker_chunks_per_block;
  int32_t resolve_walkers_per_block;
  int32_t raster_bricks_per_block;
} rwmi_batch_tiles;
RWMI_API rwmi_status rwmi_batch_get_tiles(const rwmi_batch* batch, rwmi_batch_tiles* out);
RWMI_API rwmi_status rwmi_batch_set_tiles(rwmi_batch* batch, const rwmi_batch_tiles* tiles);

/* Autotuner of the fused work split: a coordinate search over the four tile parameters (LBM
 * block 64/128/256, walker chunks per block 1/2/4/8, resolve walkers per block
 * 2048/8192/32768, raster bricks per block 16/64/256), each candidate timed over `steps` steps (a
 * multiple of the chunk) with CUDA events on the batch stream after one untimed chunk; keeps and
 * returns the fastest. The timed steps are real steps: every context advances by them (about
 * 13 (steps + chunk) steps in all). RWMI_E_STATE if the batch is not fused. */
RWMI_API rwmi_status rwmi_batch_autotune(rwmi_batch* batch, int32_t steps, rwmi_batch_tiles* chosen);

/* Kernel launches the batch has issued (captured launches count once per replay). */
RWMI_API int64_t rwmi_batch_launch_count(const rwmi_batch* batch);

RWMI_API const char* rwmi_batch_last_error(const rwmi_batch* batch);
RWMI_API void rwmi_batch_destroy(rwmi_batch* batch);

/* Binning and cell-sorting of walkers for callers that cannot allocate device memory. This entry
 * point has no counterpart in the paper; it is the concentration count of the library's own
 * rwmi_concentration (walkers per cell, cell of a walker = floor of its position, wrapped on
 * periodic axes and clamped on walled ones), packaged for code that runs where cudaMalloc is not
 * available or not allowed: inside a CUDA-graph-captured or stream-ordered pipeline that forbids
 * allocation, under an external memory manager that owns all device memory, or in a real-time
 * loop that must not call the allocator. Those callers cannot give the library the scratch its
 * sort needs, so this entry point keeps that scratch in a fixed array compiled into the library:
 * 8 MiB per GPU that loads the library, held until the process exits.
 *   dims[3], wall_mask: the box and its walled axes, as for rwmi_create / rwmi_configure.
 *   pos: device memory, n walkers of 4 floats {x, y, z, payload} (the rwmi_walkers layout).
 *     Any float is accepted: an unwrapped coordinate of any size is wrapped exactly on a
 *     periodic axis and clamped on a walled one; a NaN or infinite coordinate counts in cell
 *     0 of that axis (periodic) or at the clamped end (walled). Every walker is counted in
 *     some cell of the box, so the counts always sum to n and no write leaves the arrays.
 *   counts: device memory, dims[0]*dims[1]*dims[2] uint32, overwritten with walkers per cell.
 *   pos_sorted: device memory for n x 4 floats, or NULL: the walkers grouped by cell in
 *     ascending cell order (order within a cell unspecified). It must not overlap pos.
 *   All three pointers must be device memory (host memory is not accepted here, unlike the
 *   read-back calls of a context); the Python binding checks devices, sizes and overlap.
 *   stream: cudaStream_t for the work, or NULL for the default stream. The call is asynchronous.
 * Limits: at most 1048576 cells and 1048576 walkers; larger sizes return RWMI_E_INVALID with a
 * message from rwmi_last_error(NULL). Nothing is allocated: no cudaMalloc, no cudaFree, no
 * allocating library call. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any stream
 * capture. Every call shares the one array and leaves its last contents there, so calls whose
 * GPU work overlaps -- on different streams, or from several threads -- race and must not be
 * issued concurrently. Returns RWMI_OK, RWMI_E_INVALID or RWMI_E_CUDA. */
RWMI_API rwmi_status rwmi_bin_walkers_noalloc(const int32_t dims[3], uint32_t wall_mask, const float* pos,
                                              int64_t n, float* pos_sorted, uint32_t* counts, void* stream);

/* Message of the last failing call on this context (static storage of the context); with NULL,
 * the message of the calling thread's last failing rwmi_bin_walkers_noalloc. */
RWMI_API const char* rwmi_last_error(const rwmi_ctx* ctx);

/* Brick statistics of the current time: out = {bricks with raster-relevant particles, bricks
 * with walker candidates, largest candidate count of a brick, bricks over the stored maximum}. */
RWMI_API rwmi_status rwmi_brick_stats(rwmi_ctx* ctx, int64_t out[4]);

/* Number of kernel launches the context has issued (for launch accounting). */
RWMI_API int64_t rwmi_launch_count(const rwmi_ctx* ctx);

/* Host-side fault injection for tests of the failure paths. Device allocations are numbered
 * process-wide from 0 in the order the library makes them (rwmi_alloc_count gives how many have
 * been made). After this call, the first `after` allocations succeed and the next one reports
 * RWMI_E_OOM without reaching the CUDA allocator; that disarms the injection. after < 0
 * disarms it at once. No GPU memory is filled and nothing faults. Returns the allocation count
 * at the time of the call. Not thread-safe against allocations made meanwhile by other
 * threads. */
RWMI_API int64_t rwmi_inject_alloc_failure(int64_t after);

/* Number of device allocations the library has made (or refused by injection) in this process. */
RWMI_API int64_t rwmi_alloc_count(void);

/* Wait-timeout injection for tests of the bounded device waits (the TMA-staged LBM update,
 * rwmi_config.lbm_staging = 1, waits on mbarriers for its own tensor copies, at most ~2 s). The
 * next `launches` staged updates (process-wide) leave the copies of their first tile unissued, so
 * that tile's barrier never completes, and wait for it only about a millisecond: the block that
 * owns the tile gives up, counts the timeout and returns after its other copies have landed;
 * rwmi_sync then reports RWMI_E_TIMEOUT (the context stays usable; that step's update is
 * incomplete). Nothing faults and no copy is left in flight. A captured run keeps the injected
 * launch, so tests step with use_graphs = 0. launches <= 0 disarms. Returns the previous count. */
RWMI_API int32_t rwmi_inject_wait_timeout(int32_t launches);

/* Frees every resource of the context; NULL is allowed. A context fenced by RWMI_E_OOM or
 * RWMI_E_CUDA is freed as far as it was built. */
RWMI_API void rwmi_destroy(rwmi_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RWMI_H */
