"""Seeded synthetic inputs for the RW-MI-DELBM fluid-solute step.

This module draws run parameters, metaball particle tables and walker start positions from
seeded numpy generators. It is the one module that feeds both the CUDA library and the CPU
oracle, so it holds none of the method's arithmetic: no metaball evaluation, no lattice
Boltzmann or random-walk step. The only geometry in it is a crude bound used to keep randomly
placed particles apart (every point where a metaball of Eq. 3 reaches 1 lies within
sqrt(sum k_i) of one of its control points, by the weighted pigeonhole argument on the sum).

Workloads (the paper's experiments are stand-ins, see the docstrings):
  parity_single   -- 32^3 periodic box, one single-centre metaball (k=36, radius 6), 1e4 walkers.
  oscillator      -- 256^3 box with no-slip z-walls, 64 rigid metaball particles of 4-8 centres
                     oscillating along x, sinusoidal body force, 1e7 walkers (stand-in for the
                     Section 4 oscillator case, whose particle shapes are not published).
  precision       -- the parity_single physics scaled to 384^3 with 128 particles, 3e7 walkers.
  ragged          -- small odd-sized boxes used by the parity tests (several tiles plus a tail).
  point_source    -- Section 3.1 validation: walkers released at one point, no particles.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional
import math

import numpy as np


@dataclass
class Metaballs:
    """Rigid metaball particles (Eq. 3) on prescribed sinusoidal trajectories.

    Particle p owns control points center_offsets[p] .. center_offsets[p+1]-1. Body-frame
    control-point positions are relative to the particle origin. The origin follows
    o_p(t) = origin_p + amplitude_p * sin(2*pi*t/period_p + phase_p) (static if period_p == 0),
    and the body spins at the constant angular velocity omega_p (rad per step).
    """
    center_offsets: np.ndarray   # int32 [P+1]
    centers_body: np.ndarray     # float32 [Nc, 3]
    k: np.ndarray                # float32 [Nc]
    origin: np.ndarray           # float64 [P, 3]
    amplitude: np.ndarray        # float64 [P, 3]
    period: np.ndarray           # float64 [P]
    phase: np.ndarray            # float64 [P]
    omega: np.ndarray            # float64 [P, 3]

    @property
    def n_particles(self) -> int:
        return int(len(self.center_offsets) - 1)

    @property
    def n_centers(self) -> int:
        return int(self.center_offsets[-1])


@dataclass
class Dem:
    """Free DEM set-up (Eqs. 4-11), lattice units. The particles then move under gravity, contact
    forces and (with hydro = 1) the fluid's force and torque, instead of following prescribed
    trajectories; the prescribed motion only gives the start (origin, and velocity and spin when
    these are None). Mass and inertia follow from each metaball and its density.

    Contact law: normal stiffness kn and damping eta_n, tangential stiffness kt and damping
    eta_t, static friction mu_s; sphere_radius is the sphero-metaball's R_s per particle.
    `substeps` DEM steps make one LBM step."""
    density: object                      # float or float64 [P], relative to the fluid's rho0
    sphere_radius: np.ndarray            # float64 [P]
    velocity: Optional[np.ndarray] = None  # float64 [P, 3]
    spin: Optional[np.ndarray] = None      # float64 [P, 3]
    kn: float = 200.0
    eta_n: float = 0.0
    kt: float = 0.0
    eta_t: float = 0.0
    mu_s: float = 0.0
    gravity: tuple = (0.0, 0.0, 0.0)
    substeps: int = 10
    hydro: int = 1


@dataclass
class Workload:
    name: str
    dims: tuple                          # (nx, ny, nz)
    tau: float
    D: float                             # walker diffusion coefficient, lattice units
    seed: int                            # Philox key for walker noise and seeding
    q: int = 15                          # 15 (D3Q15) or 19 (D3Q19)
    wall_mask: int = 0                   # bit 0/1/2: no-slip walls on the x/y/z faces
    body_force: tuple = (0.0, 0.0, 0.0)  # force density F0 (lattice units)
    force_period: float = 0.0            # F(t) = F0 sin(2 pi t / period); 0 -> constant F0
    rho0: float = 1.0
    init_velocity: tuple = (0.0, 0.0, 0.0)
    metaballs: Optional[Metaballs] = None
    n_walkers: int = 0
    walker_box: Optional[tuple] = None   # ((lo3), (hi3)) for uniform seeding in the fluid
    walker_positions: Optional[np.ndarray] = None  # explicit float32 [N, 3] start positions
    steps: int = 1
    storage: int = 1                     # 0 FP32, 1 FP32 shifted by w_i rho0, 2 FP16 shifted, 3 FP64 shifted
    sort_interval: int = 0
    moment_interval: int = 0
    coupling: int = 0                    # 0 partially saturated cells, 1 IBB (Section 2.4.3)
    dem: Optional[Dem] = None            # free DEM instead of prescribed trajectories
    notes: str = ""

    @property
    def n_cells(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])


def empty_metaballs() -> Metaballs:
    return Metaballs(
        center_offsets=np.zeros(1, np.int32),
        centers_body=np.zeros((0, 3), np.float32),
        k=np.zeros(0, np.float32),
        origin=np.zeros((0, 3)), amplitude=np.zeros((0, 3)),
        period=np.zeros(0), phase=np.zeros(0), omega=np.zeros((0, 3)))


def placement_radius(centers_body: np.ndarray, k: np.ndarray) -> float:
    """Crude bound on a particle's extent: max |c_i| + sqrt(sum k_i). Placement only."""
    if len(k) == 0:
        return 0.0
    return float(np.max(np.linalg.norm(centers_body.astype(np.float64), axis=1))
                 + np.sqrt(np.sum(k.astype(np.float64))))


def random_metaballs(rng: np.random.Generator, n_particles: int, dims, wall_mask: int,
                     n_centers=(4, 8), sigma=4.0, k_range=(20.0, 60.0),
                     amplitude=(0.0, 0.0, 0.0), period=0.0, phase=0.0,
                     omega=(0.0, 0.0, 0.0), max_tries=100000) -> Metaballs:
    """Random non-overlapping metaball particles.

    Each particle has U{n_centers} control points drawn from N(0, sigma^2 I) about its origin
    and weights k ~ U[k_range]. Origins are placed by random sequential addition with the crude
    placement_radius bound as a hard-sphere radius (minimum image on periodic axes). All
    particles share one drive (amplitude, period, phase), so their relative positions never
    change and non-overlap holds for the whole trajectory. Along a walled axis the particle
    keeps clear of the wall by its radius plus one cell plus the drive amplitude on that axis.
    """
    dims = np.asarray(dims, np.float64)
    amp = np.asarray(amplitude, np.float64)
    cb_list, k_list, rad = [], [], []
    for _ in range(n_particles):
        nc = int(rng.integers(n_centers[0], n_centers[1] + 1))
        cb_list.append(rng.normal(0.0, sigma, size=(nc, 3)).astype(np.float32))
        k_list.append(rng.uniform(k_range[0], k_range[1], size=nc).astype(np.float32))
        rad.append(placement_radius(cb_list[-1], k_list[-1]))
    # Largest first: random sequential addition packs far better that way.
    order = np.argsort(-np.asarray(rad), kind="stable")
    cb_list = [cb_list[i] for i in order]
    k_list = [k_list[i] for i in order]
    rad = [rad[i] for i in order]
    origins = []
    for p in range(n_particles):
        lo = np.zeros(3)
        hi = dims.copy()
        for a in range(3):
            if wall_mask >> a & 1:
                lo[a] = rad[p] + 1.0 + abs(amp[a])
                hi[a] = dims[a] - rad[p] - 1.0 - abs(amp[a])
                if hi[a] <= lo[a]:
                    raise ValueError("particle does not fit between the walls")
        for _try in range(max_tries):
            o = lo + rng.random(3) * (hi - lo)
            ok = True
            for qq, oq in enumerate(origins):
                d = o - oq
                for a in range(3):
                    if not (wall_mask >> a & 1):
                        d[a] -= dims[a] * np.round(d[a] / dims[a])
                if np.linalg.norm(d) < rad[p] + rad[qq] + 1.0:
                    ok = False
                    break
            if ok:
                origins.append(o)
                break
        else:
            raise RuntimeError("random placement failed; box too crowded")
    offs = np.zeros(n_particles + 1, np.int32)
    offs[1:] = np.cumsum([len(c) for c in cb_list])
    P = n_particles
    return Metaballs(
        center_offsets=offs,
        centers_body=np.concatenate(cb_list).astype(np.float32) if P else np.zeros((0, 3), np.float32),
        k=np.concatenate(k_list).astype(np.float32) if P else np.zeros(0, np.float32),
        origin=np.array(origins, np.float64).reshape(P, 3),
        amplitude=np.tile(amp, (P, 1)),
        period=np.full(P, float(period)),
        phase=np.full(P, float(phase)),
        omega=np.tile(np.asarray(omega, np.float64), (P, 1)))


def single_sphere(center, k=36.0) -> Metaballs:
    """One static particle with a single control point: the surface is a sphere of radius sqrt(k)."""
    return Metaballs(
        center_offsets=np.array([0, 1], np.int32),
        centers_body=np.zeros((1, 3), np.float32),
        k=np.array([k], np.float32),
        origin=np.array([center], np.float64),
        amplitude=np.zeros((1, 3)), period=np.zeros(1), phase=np.zeros(1),
        omega=np.zeros((1, 3)))


def parity_single(steps: int = 500, n_walkers: int = 10_000, q: int = 15) -> Workload:
    """Plain-method parity case: D3Q15 BGK, periodic 32^3, tau 0.8, constant body force 1e-6
    along x, one stationary single-centre metaball (k=36, radius 6) at the box centre,
    1e4 walkers uniform in the fluid, D=0.01, 500 steps, Philox seed 0."""
    return Workload(
        name="parity_single_32", dims=(32, 32, 32), tau=0.8, D=0.01, seed=0, q=q,
        body_force=(1e-6, 0.0, 0.0), metaballs=single_sphere((16.0, 16.0, 16.0), 36.0),
        n_walkers=n_walkers, walker_box=((0.0, 0.0, 0.0), (32.0, 32.0, 32.0)), steps=steps)


def oscillator(n: int = 256, n_particles: int = 64, n_walkers: int = 10_000_000,
               steps: int = 20000, morph_seed: int = 1, seed: int = 1, q: int = 15,
               storage: int = 1) -> Workload:
    """Oscillator stand-in for the Section 4 shaking-bath case (Eq. 37 drives the particles).

    n^3 box, no-slip z-walls, body force 5e-6 sin(2 pi t/2000) along x, tau 0.7; 64 rigid
    particles of 4-8 centres (N(0, 4^2) about the origin, k ~ U[20, 60]) placed at random
    without overlap, all translating as 5 sin(2 pi t/2000) along x; 1e7 walkers uniform in the
    fluid, D=0.005. The particle morphologies A-D and the cobblestone scans are not published,
    so random metaball clusters stand in for them.
    """
    rng = np.random.default_rng(morph_seed)
    mb = random_metaballs(rng, n_particles, (n, n, n), wall_mask=4, amplitude=(5.0, 0.0, 0.0),
                          period=2000.0)
    return Workload(
        name=f"oscillator_{n}", dims=(n, n, n), tau=0.7, D=0.005, seed=seed, q=q, wall_mask=4,
        body_force=(5e-6, 0.0, 0.0), force_period=2000.0, metaballs=mb, n_walkers=n_walkers,
        walker_box=((0.0, 0.0, 0.0), (float(n), float(n), float(n))), steps=steps,
        storage=storage)


def precision(n: int = 384, n_particles: int = 128, n_walkers: int = 30_000_000,
              seed: int = 2, storage: int = 1) -> Workload:
    """Precision case: the parity_single physics (periodic, tau 0.8, F=1e-6 x) at n^3 with
    randomly placed static particles and 3e7 walkers."""
    rng = np.random.default_rng(seed)
    mb = random_metaballs(rng, n_particles, (n, n, n), wall_mask=0)
    return Workload(
        name=f"precision_{n}", dims=(n, n, n), tau=0.8, D=0.01, seed=seed,
        body_force=(1e-6, 0.0, 0.0), metaballs=mb, n_walkers=n_walkers,
        walker_box=((0.0, 0.0, 0.0), (float(n),) * 3), steps=20, storage=storage)


def ragged(dims=(40, 36, 26), n_particles: int = 3, n_walkers: int = 3000, seed: int = 7,
           walls: int = 4, q: int = 15, moving: bool = True, storage: int = 1,
           k_range=(4.0, 9.0), n_centers=(2, 3), sigma=1.0) -> Workload:
    """Small odd-sized box with a few moving multi-centre particles; spans several tiles of
    every kernel and leaves a ragged tail."""
    rng = np.random.default_rng(seed)
    # drive speeds stay below 0.07 lattice units (low Mach number): 1.5 * 2 pi / 150 = 0.063
    mb = random_metaballs(rng, n_particles, dims, wall_mask=walls, n_centers=n_centers,
                          sigma=sigma, k_range=k_range,
                          amplitude=(1.5, 0.75, 0.0) if moving else (0.0, 0.0, 0.0),
                          period=150.0 if moving else 0.0, phase=0.3,
                          omega=(0.0, 0.0, 0.004) if moving else (0.0, 0.0, 0.0))
    return Workload(
        name=f"ragged_{dims[0]}x{dims[1]}x{dims[2]}", dims=tuple(dims), tau=0.75, D=0.02,
        seed=seed, q=q, wall_mask=walls, body_force=(2e-5, 5e-6, 0.0), force_period=60.0,
        metaballs=mb, n_walkers=n_walkers, walker_box=((0.0, 0.0, 0.0), tuple(float(d) for d in dims)),
        steps=30, storage=storage)


def point_source(n: int = 100, n_walkers: int = 1_000_000, D: float = 0.2,
                 velocity=(0.0, 0.0, 0.0), steps: int = 100, seed: int = 3) -> Workload:
    """Section 3.1 validation: a point source of walkers at the box centre in a quiescent or
    uniformly moving periodic fluid. The paper's setting (D = 1e-3 m^2/s, dx = 1e-3 m,
    dt = 2e-4 s, u = 1 m/s) is D = 0.2 and u = 0.2 in lattice units."""
    pos = np.full((n_walkers, 3), n / 2.0, np.float32)
    return Workload(
        name=f"point_source_{n}", dims=(n, n, n), tau=1.0, D=D, seed=seed,
        init_velocity=tuple(velocity), metaballs=empty_metaballs(), n_walkers=n_walkers,
        walker_positions=pos, steps=steps)


def _fitting_metaballs(rng, n_particles, dims, wall_mask, **kw) -> Metaballs:
    """random_metaballs with one particle fewer each time the box is too crowded."""
    while True:
        try:
            return random_metaballs(rng, n_particles, dims, wall_mask, max_tries=2000, **kw)
        except RuntimeError:
            if n_particles <= 1:
                raise
            n_particles -= 1


def batched(n_domains: int = 64, seed: int = 3, edge=(48, 160), particles=(4, 32),
            centers=(2, 10), walkers=(100_000, 2_000_000), tau=(0.6, 1.0), D=(0.001, 0.02),
            steps: int = 1000, q: int = 15, storage: int = 1, sort_interval: int = 16,
            walker_scale: float = 1.0) -> list:
    """Many independent periodic domains of different sizes advanced together.

    Per domain: cubic edge ~ U{edge}; particle count from U{particles}, scaled down with the
    box volume relative to the largest edge (a 48^3 box cannot hold 32 clusters), at least the
    lower bound; U{centers} control points per particle (N(0, 1.5^2 I), k ~ U[4, 16]); walkers
    ~ U[walkers] (times walker_scale); tau ~ U[tau]; D ~ U[D]; constant body force 1e-6 along
    x as in the single-particle case; particles translate 2 sin(2 pi t / 1000) along x with
    random phase per domain. All domains share sort_interval, so their step chunks line up.
    """
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n_domains):
        n = int(rng.integers(edge[0], edge[1] + 1))
        frac = (n / float(edge[1])) ** 3
        n_p = int(rng.integers(particles[0], particles[1] + 1))
        n_p = max(particles[0], int(round(n_p * frac)))
        mb = _fitting_metaballs(rng, n_p, (n, n, n), 0, n_centers=centers, sigma=1.5,
                                k_range=(4.0, 16.0), amplitude=(2.0, 0.0, 0.0), period=1000.0,
                                phase=float(rng.uniform(0.0, 2.0 * np.pi)))
        nw = int(round(rng.uniform(walkers[0], walkers[1]) * walker_scale))
        out.append(Workload(
            name=f"batched_{d}_{n}", dims=(n, n, n), tau=float(rng.uniform(*tau)),
            D=float(rng.uniform(*D)), seed=seed * 1000 + d, q=q, body_force=(1e-6, 0.0, 0.0),
            metaballs=mb, n_walkers=nw, walker_box=((0.0, 0.0, 0.0), (float(n),) * 3),
            steps=steps, storage=storage, sort_interval=sort_interval))
    return out


@dataclass
class Request:
    """One simulation request of the served stream."""
    rid: int
    arrival: float       # seconds after the stream starts
    workload: Workload


def served(n_requests: int = 64, rate: float = 20.0, seed: int = 4, edge=(32, 256),
           walkers=(100_000, 10_000_000), steps=(1000, 20000), storage=(1, 2),
           step_scale: float = 1.0, walker_scale: float = 1.0, sort_interval: int = 16) -> list:
    """Poisson stream of simulation requests (mean `rate` per second).

    Per request: exponential inter-arrival gap with mean 1/rate; cubic edge log-uniform in
    [edge]; walkers log-uniform in [walkers] (times walker_scale, at most 2 per cell); steps
    uniform in [steps] (times step_scale, rounded to a multiple of sort_interval); storage
    picked from `storage` (FP32-shift or FP16-shift); a random single-particle-style
    morphology: 1-4 metaball clusters (fewer in boxes below 64^3) of 1-6 centres (k ~ U[20, 60],
    sigma 3, both scaled down by (n/64)^2 and n/64 below 64^3) at rest, periodic
    box, tau ~ U[0.6, 1.0], D ~ U[0.001, 0.02], constant body force 1e-6 along x.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(np.exp(rng.uniform(np.log(edge[0]), np.log(edge[1])))))
        nw = int(round(np.exp(rng.uniform(np.log(walkers[0]), np.log(walkers[1]))) * walker_scale))
        nw = max(1, min(nw, 2 * n ** 3))
        ns = int(rng.integers(steps[0], steps[1] + 1) * step_scale)
        ns = max(sort_interval, ns - ns % sort_interval)
        st = int(storage[int(rng.integers(0, len(storage)))])
        n_p = int(rng.integers(1, 5))
        n_p = max(1, min(n_p, int(round(n_p * (n / 64.0) ** 3))))
        ks = min(1.0, (n / 64.0) ** 2)
        mb = _fitting_metaballs(rng, n_p, (n, n, n), 0, n_centers=(1, 6), sigma=3.0 * math.sqrt(ks),
                                k_range=(20.0 * ks, 60.0 * ks))
        w = Workload(
            name=f"request_{r}_{n}", dims=(n, n, n), tau=float(rng.uniform(0.6, 1.0)),
            D=float(rng.uniform(0.001, 0.02)), seed=seed * 100000 + r, body_force=(1e-6, 0.0, 0.0),
            metaballs=mb, n_walkers=nw, walker_box=((0.0, 0.0, 0.0), (float(n),) * 3), steps=ns,
            storage=st, sort_interval=sort_interval)
        reqs.append(Request(r, t, w))
    return reqs


def with_(w: Workload, **kw) -> Workload:
    return replace(w, **kw)


# ------------------------------------------------------------------------------------------
# Free-DEM inputs
# ------------------------------------------------------------------------------------------
def sphere_radii(mb: Metaballs, fraction: float = 0.5) -> np.ndarray:
    """R_s of each particle: a fraction of its smallest control-point radius sqrt(k_i). Every
    such sphere lies inside the particle, so R_s stays below the bound radius."""
    out = np.zeros(mb.n_particles)
    for p in range(mb.n_particles):
        sl = slice(int(mb.center_offsets[p]), int(mb.center_offsets[p + 1]))
        out[p] = fraction * float(np.sqrt(mb.k[sl].astype(np.float64)).min())
    return out


def dem_box(dims=(40, 36, 44), n_particles: int = 4, seed: int = 11, density: float = 2.5,
            speed: float = 0.05, gravity=(0.0, 0.0, -5e-4), kn: float = 50.0, eta_n: float = 2.0,
            kt: float = 20.0, eta_t: float = 1.0, mu_s: float = 0.4, substeps: int = 10,
            hydro: int = 1, n_walkers: int = 3000, storage: int = 1, q: int = 15) -> Workload:
    """Small walled box (z-walls) of free multi-centre particles: random start velocities of the
    given speed, gravity along -z, damped frictional contacts; several contacts within a few
    tens of steps. Parity and invariant tests use it."""
    rng = np.random.default_rng(seed)
    mb = random_metaballs(rng, n_particles, dims, wall_mask=4, n_centers=(2, 3), sigma=1.2,
                          k_range=(4.0, 9.0))
    v = rng.normal(size=(n_particles, 3))
    v *= speed / np.linalg.norm(v, axis=1, keepdims=True)
    w = rng.normal(scale=0.01, size=(n_particles, 3))
    dem = Dem(density=density, sphere_radius=sphere_radii(mb), velocity=v, spin=w, kn=kn,
              eta_n=eta_n, kt=kt, eta_t=eta_t, mu_s=mu_s, gravity=tuple(gravity), substeps=substeps,
              hydro=hydro)
    return Workload(
        name=f"dem_box_{dims[0]}x{dims[1]}x{dims[2]}", dims=tuple(dims), tau=0.8, D=0.02, seed=seed, q=q,
        wall_mask=4, metaballs=mb, dem=dem, n_walkers=n_walkers,
        walker_box=((0.0, 0.0, 0.0), tuple(float(d) for d in dims)), steps=40, storage=storage)


def oscillator_dem(n: int = 256, n_particles: int = 64, n_walkers: int = 10_000_000, density: float = 2.0,
                   gravity=(0.0, 0.0, -2e-5), kn: float = 1000.0, eta_n: float = 20.0, kt: float = 400.0,
                   eta_t: float = 10.0, mu_s: float = 0.5, substeps: int = 10, **kw) -> Workload:
    """The oscillator workload with free particles: they start on their prescribed motion
    (x-velocity 5 (2 pi / 2000)) and then move under the oscillating flow, gravity and
    contacts."""
    w = oscillator(n=n, n_particles=n_particles, n_walkers=n_walkers, **kw)
    dem = Dem(density=density, sphere_radius=sphere_radii(w.metaballs), kn=kn, eta_n=eta_n, kt=kt,
              eta_t=eta_t, mu_s=mu_s, gravity=tuple(gravity), substeps=substeps, hydro=1)
    return replace(w, name=f"oscillator_dem_{n}", dem=dem)
