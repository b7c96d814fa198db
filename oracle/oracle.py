"""ctypes shim over the FP64 C oracle (rwmi_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline
leg use this module; the product path never does. It imports nothing from the CUDA package.
Workload objects are read by attribute (duck typing), so the shared seeded input module is the
only thing both sides see.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rwmi_oracle.c")
# RWMI_ORACLE_LIB names a prebuilt oracle library to load instead (tests/mutation_check.py builds
# deliberately broken copies elsewhere and runs the pins against them)
_PREBUILT = os.environ.get("RWMI_ORACLE_LIB")
_LIB = _PREBUILT or os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: the binary32 decisions must round exactly as written (no fused multiply-add)
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds). Rebuilt when the source is newer than the library."""
    if _PREBUILT:
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = P
            L.orc_create.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_double, C.c_double, C.c_uint64,
                                     C.c_int, dp, C.c_double, C.c_double, dp]
            L.orc_destroy.argtypes = [P]
            L.orc_set_metaballs.argtypes = [P, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_seed_walkers.restype = C.c_longlong
            L.orc_seed_walkers.argtypes = [P, C.c_longlong, dp, dp, C.c_int]
            L.orc_set_walkers.argtypes = [P, C.c_longlong, C.c_void_p, C.c_void_p]
            L.orc_step.argtypes = [P, C.c_longlong]
            L.orc_step_fluid.argtypes = [P, C.c_longlong]
            L.orc_time.restype = C.c_longlong
            L.orc_time.argtypes = [P]
            L.orc_set_time.argtypes = [P, C.c_longlong]
            for name in ("orc_velocity", "orc_density", "orc_populations", "orc_set_populations",
                         "orc_set_velocity", "orc_concentration", "orc_moments",
                         "orc_mass_momentum", "orc_forces", "orc_counters"):
                getattr(L, name).argtypes = [P, C.c_void_p]
            L.orc_solid.argtypes = [P, C.c_longlong, C.c_void_p, C.c_void_p]
            L.orc_solid_cells.argtypes = [P, C.c_longlong, C.c_longlong, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
            L.orc_walkers.argtypes = [P, C.c_void_p, C.c_void_p]
            L.orc_bin_positions.argtypes = [P, C.c_longlong, C.c_void_p, C.c_void_p]
            L.orc_lbm_cells.argtypes = [P, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_walkers_advance.argtypes = [P, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_philox.argtypes = [C.c_uint64, C.c_void_p, C.c_void_p]
            L.orc_step_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_void_p]
            L.orc_philox_find_seed.restype = C.c_longlong
            L.orc_philox_find_seed.argtypes = [C.c_uint64, C.c_longlong, C.c_void_p, C.c_int, C.c_uint32]
            L.orc_metaball.restype = C.c_double
            L.orc_metaball.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_metaball32.restype = C.c_float
            L.orc_metaball32.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p]
            L.orc_bound_radius.restype = C.c_double
            L.orc_bound_radius.argtypes = [P, C.c_int]
            L.orc_inside.restype = C.c_int
            L.orc_inside.argtypes = [P, C.c_longlong, C.c_void_p]
            L.orc_bisect.restype = C.c_int
            L.orc_bisect.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_reflect.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_refill.restype = C.c_int
            L.orc_refill.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p, C.c_uint32, C.c_void_p]
            L.orc_trilinear.argtypes = [P, C.c_void_p, C.c_void_p]
            L.orc_pose.argtypes = [P, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_lattice.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
            L.orc_set_coupling.argtypes = [P, C.c_int]
            L.orc_nodes.argtypes = [P, C.c_longlong, C.c_void_p]
            L.orc_ibb_q.restype = C.c_double
            L.orc_ibb_q.argtypes = [P, C.c_longlong, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong, C.c_void_p]
            L.orc_set_dem.restype = C.c_int
            L.orc_set_dem.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, dp,
                                      C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            for name in ("orc_particle_state", "orc_set_particle_state", "orc_dem_mass"):
                getattr(L, name).argtypes = [P, C.c_void_p]
            L.orc_dem_pair_geom.argtypes = [P, C.c_int, C.c_int, C.c_void_p]
            L.orc_dem_wall_geom.argtypes = [P, C.c_int, C.c_int, C.c_void_p]
            L.orc_dem_contact_force.argtypes = [P, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_double, C.c_void_p, C.c_void_p]
            L.orc_dem_advance.argtypes = [P, C.c_longlong]
            L.orc_set_prev_nodes.argtypes = [P, C.c_longlong, C.c_void_p]
            L.orc_ibb_link.restype = C.c_double
            L.orc_ibb_link.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp, dp, dp, C.c_double]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _d3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def philox(seed: int, ctr) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(C.c_uint64(seed), _ptr(c), _ptr(out))
    return out


def step_normals(seed: int, walker_id: int, t: int) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_step_normals(C.c_uint64(seed), C.c_uint32(walker_id), C.c_uint32(t), _ptr(out))
    return out


def philox_find_seed(seed0: int, count: int, ctr, word: int, target: int) -> int:
    """First seed in [seed0, seed0 + count) whose Philox word `word` for counter ctr has
    (word >> 8) == target, or -1 (test helper)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    return int(lib().orc_philox_find_seed(C.c_uint64(seed0), int(count), _ptr(c), int(word), C.c_uint32(target)))


def lattice(q: int):
    e = np.zeros((q, 3), np.int32)
    w = np.zeros(q)
    lib().orc_lattice(q, _ptr(e), _ptr(w))
    return e, w


class Oracle:
    """One oracle simulation context (FP64 state on the host)."""

    def __init__(self, dims, q=15, tau=0.8, D=0.01, seed=0, wall_mask=0, body_force=(0, 0, 0),
                 force_period=0.0, rho0=1.0, init_velocity=(0, 0, 0)):
        L = lib()
        d = (C.c_int * 3)(*[int(x) for x in dims])
        self.dims = tuple(int(x) for x in dims)
        self.q = int(q)
        self.n_cells = self.dims[0] * self.dims[1] * self.dims[2]
        self.h = L.orc_create(d, int(q), float(tau), float(D), C.c_uint64(int(seed)), int(wall_mask),
                              _d3(body_force), float(force_period), float(rho0), _d3(init_velocity))
        if not self.h:
            raise ValueError("oracle: bad configuration")
        self.n_particles = 0
        self.n_walkers = 0

    @classmethod
    def from_workload(cls, w, seed_walkers: bool = True) -> "Oracle":
        o = cls(w.dims, q=w.q, tau=w.tau, D=w.D, seed=w.seed, wall_mask=w.wall_mask,
                body_force=w.body_force, force_period=w.force_period, rho0=w.rho0,
                init_velocity=w.init_velocity)
        if getattr(w, "coupling", 0):
            o.set_coupling(w.coupling)
        if w.metaballs is not None and w.metaballs.n_particles > 0:
            o.set_metaballs(w.metaballs)
            if getattr(w, "dem", None) is not None:
                o.set_dem(w.dem)
        if seed_walkers and w.n_walkers:
            if w.walker_positions is not None:
                o.set_walkers(np.asarray(w.walker_positions, np.float64))
            else:
                lo, hi = w.walker_box
                fails = o.seed_walkers(w.n_walkers, lo, hi)
                if fails:
                    raise RuntimeError(f"oracle seeding: {fails} walkers found no free point")
        return o

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    # ---- setup ----
    def set_metaballs(self, mb):
        self._mb = dict(
            coff=np.ascontiguousarray(mb.center_offsets, np.int32),
            cb=np.ascontiguousarray(mb.centers_body, np.float32).reshape(-1),
            k=np.ascontiguousarray(mb.k, np.float32),
            org=np.ascontiguousarray(mb.origin, np.float64).reshape(-1),
            amp=np.ascontiguousarray(mb.amplitude, np.float64).reshape(-1),
            per=np.ascontiguousarray(mb.period, np.float64),
            pha=np.ascontiguousarray(mb.phase, np.float64),
            omg=np.ascontiguousarray(mb.omega, np.float64).reshape(-1))
        m = self._mb
        self.n_particles = int(len(m["coff"]) - 1)
        lib().orc_set_metaballs(self.h, self.n_particles, _ptr(m["coff"]), _ptr(m["cb"]), _ptr(m["k"]),
                                _ptr(m["org"]), _ptr(m["amp"]), _ptr(m["per"]), _ptr(m["pha"]), _ptr(m["omg"]))

    def set_dem(self, dem):
        """Free DEM (Eqs. 4-11) instead of the prescribed trajectories, from the current time."""
        P = self.n_particles
        self._dem = dict(
            rho=np.ascontiguousarray(np.broadcast_to(dem.density, (P,)), np.float64),
            Rs=np.ascontiguousarray(dem.sphere_radius, np.float64).reshape(P),
            v=None if dem.velocity is None else np.ascontiguousarray(dem.velocity, np.float64).reshape(P * 3),
            w=None if dem.spin is None else np.ascontiguousarray(dem.spin, np.float64).reshape(P * 3))
        d = self._dem
        rc = lib().orc_set_dem(self.h, float(dem.kn), float(dem.eta_n), float(dem.kt), float(dem.eta_t),
                               float(dem.mu_s), _d3(dem.gravity), int(dem.substeps), int(dem.hydro),
                               _ptr(d["rho"]), _ptr(d["Rs"]),
                               None if d["v"] is None else _ptr(d["v"]),
                               None if d["w"] is None else _ptr(d["w"]))
        if rc != 0:
            raise ValueError("oracle: invalid DEM set-up")

    def dem_mass(self) -> np.ndarray:
        """[P, 10]: mass, centre of mass (given body frame), inertia about it (xx yy zz xy xz yz)."""
        out = np.zeros((max(self.n_particles, 1), 10))
        lib().orc_dem_mass(self.h, _ptr(out))
        return out[: self.n_particles]

    def particle_state(self) -> np.ndarray:
        """[P, 13]: origin (unwrapped), quaternion (w, x, y, z), velocity, spin."""
        out = np.zeros((max(self.n_particles, 1), 13))
        lib().orc_particle_state(self.h, _ptr(out))
        return out[: self.n_particles]

    def set_particle_state(self, st):
        st = np.ascontiguousarray(st, np.float64).reshape(self.n_particles, 13)
        lib().orc_set_particle_state(self.h, _ptr(st))

    def dem_pair_geom(self, i, j) -> dict:
        """Eqs. 7-9 for particles i, j in the current state, as a new contact."""
        out = np.zeros(16)
        lib().orc_dem_pair_geom(self.h, int(i), int(j), _ptr(out))
        return dict(xm=out[0:3], xc0=out[3:6], xc1=out[6:9], n=out[9:12], delta=float(out[12]), xcp=out[13:16])

    def dem_wall_geom(self, p, face) -> dict:
        """Eqs. 10-11 for particle p and wall face 2 axis + side, as a new contact."""
        out = np.zeros(13)
        lib().orc_dem_wall_geom(self.h, int(p), int(face), _ptr(out))
        return dict(xcm=out[0:3], xcw=out[3:6], n=out[6:9], delta=float(out[9]), xcp=out[10:13])

    def dem_contact_force(self, delta, n, vi, vj, dt, xi):
        """The contact law with this context's DEM parameters: (force on body i, updated spring)."""
        arr = [np.ascontiguousarray(v, np.float64).reshape(3).copy() for v in (n, vi, vj, xi)]
        F = np.zeros(3)
        lib().orc_dem_contact_force(self.h, float(delta), _ptr(arr[0]), _ptr(arr[1]), _ptr(arr[2]),
                                    float(dt), _ptr(arr[3]), _ptr(F))
        return F, arr[3]

    def set_prev_nodes(self, t_prev, nodes):
        """IBB with the free DEM: node classes of t_prev, refilled from at the step t_prev + 1."""
        nodes = np.ascontiguousarray(nodes, np.int32).reshape(self.n_cells)
        lib().orc_set_prev_nodes(self.h, int(t_prev), _ptr(nodes))

    def dem_advance(self, n=1):
        """n LBM steps' worth of DEM steps, fluid and walkers frozen."""
        lib().orc_dem_advance(self.h, int(n))

    def seed_walkers(self, n, lo, hi, max_attempts=1000) -> int:
        self.n_walkers = int(n)
        return int(lib().orc_seed_walkers(self.h, int(n), _d3(lo), _d3(hi), int(max_attempts)))

    def set_walkers(self, x, x0=None):
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        self.n_walkers = len(x)
        x0p = None
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, np.float64).reshape(-1, 3)
            x0p = _ptr(x0)
        lib().orc_set_walkers(self.h, len(x), _ptr(x), x0p)

    # ---- stepping ----
    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    def step_fluid(self, n=1):
        lib().orc_step_fluid(self.h, int(n))

    @property
    def t(self) -> int:
        return int(lib().orc_time(self.h))

    def set_time(self, t):
        lib().orc_set_time(self.h, int(t))

    def set_coupling(self, mode):
        """0: partially saturated cells; 1: IBB, momentum exchange and refilling (Section 2.4.3)."""
        lib().orc_set_coupling(self.h, int(mode))

    def nodes(self, t=None):
        """IBB node classes at time t: 1 + owning particle for solid nodes, 0 for fluid."""
        out = np.zeros(self.n_cells, np.int32)
        lib().orc_nodes(self.h, int(self.t if t is None else t), _ptr(out))
        return out

    def ibb_q(self, t, p, ijk, e):
        """q of Eq. 25 on the link from node ijk along lattice vector e, particle p, time t."""
        ev = np.ascontiguousarray(e, np.int32)
        return float(lib().orc_ibb_q(self.h, int(t), int(p), int(ijk[0]), int(ijk[1]), int(ijk[2]), _ptr(ev)))

    # ---- outputs ----
    def velocity(self) -> np.ndarray:
        out = np.zeros((self.n_cells, 3))
        lib().orc_velocity(self.h, _ptr(out))
        return out

    def density(self) -> np.ndarray:
        out = np.zeros(self.n_cells)
        lib().orc_density(self.h, _ptr(out))
        return out

    def populations(self) -> np.ndarray:
        out = np.zeros((self.q, self.n_cells))
        lib().orc_populations(self.h, _ptr(out))
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64).reshape(self.q, self.n_cells)
        lib().orc_set_populations(self.h, _ptr(f))

    def set_velocity(self, u):
        u = np.ascontiguousarray(u, np.float64).reshape(self.n_cells, 3)
        lib().orc_set_velocity(self.h, _ptr(u))

    def solid(self, t=None):
        t = self.t if t is None else int(t)
        cnt = np.zeros(self.n_cells, np.int32)
        own = np.zeros(self.n_cells, np.int32)
        lib().orc_solid(self.h, t, _ptr(cnt), _ptr(own))
        return cnt, own

    def solid_cells(self, cells, t=None):
        """Solid sub-sample count and owner of the listed cells at step t (default: now)."""
        cells = np.ascontiguousarray(cells, np.int64)
        cnt = np.zeros(len(cells), np.int32)
        own = np.zeros(len(cells), np.int32)
        lib().orc_solid_cells(self.h, int(self.t if t is None else t), len(cells), _ptr(cells),
                              _ptr(cnt), _ptr(own))
        return cnt, own

    def walkers(self):
        x = np.zeros((self.n_walkers, 3))
        x0 = np.zeros((self.n_walkers, 3))
        lib().orc_walkers(self.h, _ptr(x), _ptr(x0))
        return x, x0

    def concentration(self) -> np.ndarray:
        out = np.zeros(self.n_cells, np.uint32)
        lib().orc_concentration(self.h, _ptr(out))
        return out

    def bin_positions(self, pos) -> np.ndarray:
        pos = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
        out = np.zeros(len(pos), np.int64)
        lib().orc_bin_positions(self.h, len(pos), _ptr(pos), _ptr(out))
        return out

    def moments(self) -> np.ndarray:
        out = np.zeros(13)
        lib().orc_moments(self.h, _ptr(out))
        return out

    def mass_momentum(self) -> np.ndarray:
        out = np.zeros(4)
        lib().orc_mass_momentum(self.h, _ptr(out))
        return out

    def forces(self) -> np.ndarray:
        out = np.zeros((max(self.n_particles, 1), 6))
        lib().orc_forces(self.h, _ptr(out))
        return out[: self.n_particles]

    def counters(self) -> dict:
        out = np.zeros(8, np.int64)
        lib().orc_counters(self.h, _ptr(out))
        keys = ["type_I", "type_II", "type_III", "type_IV", "bisect_fail", "refill_fail",
                "wall_fail", "seed_fail"]
        return dict(zip(keys, (int(v) for v in out)))

    # ---- sampled checks ----
    def lbm_cells(self, cells):
        cells = np.ascontiguousarray(cells, np.int64)
        n = len(cells)
        fo = np.zeros((self.q, n))
        uo = np.zeros((n, 3))
        ro = np.zeros(n)
        lib().orc_lbm_cells(self.h, n, _ptr(cells), _ptr(fo), _ptr(uo), _ptr(ro))
        return fo, uo, ro

    def walkers_advance(self, x, ids):
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        ids = np.ascontiguousarray(ids, np.uint32)
        out = np.zeros_like(x)
        lib().orc_walkers_advance(self.h, len(x), _ptr(x), _ptr(ids), _ptr(out))
        return out

    # ---- single functions ----
    def metaball(self, p, x, t=None):
        t = self.t if t is None else int(t)
        x = np.ascontiguousarray(x, np.float64)
        g = np.zeros(3)
        f = lib().orc_metaball(self.h, t, int(p), _ptr(x), _ptr(g))
        return float(f), g

    def metaball32(self, p, x, t=None):
        t = self.t if t is None else int(t)
        x = np.ascontiguousarray(x, np.float32)
        return np.float32(lib().orc_metaball32(self.h, t, int(p), _ptr(x)))

    def bound_radius(self, p) -> float:
        return float(lib().orc_bound_radius(self.h, int(p)))

    def inside(self, x, t=None) -> int:
        t = self.t if t is None else int(t)
        x = np.ascontiguousarray(x, np.float64)
        return int(lib().orc_inside(self.h, t, _ptr(x)))

    def bisect(self, p, a, b, t=None):
        t = self.t if t is None else int(t)
        a = np.ascontiguousarray(a, np.float64)
        b = np.ascontiguousarray(b, np.float64)
        xi = np.zeros(3)
        ok = lib().orc_bisect(self.h, t, int(p), _ptr(a), _ptr(b), _ptr(xi))
        return bool(ok), xi

    def reflect(self, p, xint, xf, t=None):
        t = self.t if t is None else int(t)
        xint = np.ascontiguousarray(xint, np.float64)
        xf = np.ascontiguousarray(xf, np.float64)
        out = np.zeros(3)
        lib().orc_reflect(self.h, t, int(p), _ptr(xint), _ptr(xf), _ptr(out))
        return out

    def refill(self, p, x, walker_id, t=None):
        """Refill a walker at x inside particle p; particles at t+1, noise counter (id, t, 1, 0)."""
        t = self.t if t is None else int(t)
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros(3)
        ok = lib().orc_refill(self.h, t, int(p), _ptr(x), C.c_uint32(walker_id), _ptr(out))
        return bool(ok), out

    def trilinear(self, x):
        x = np.ascontiguousarray(x, np.float64)
        out = np.zeros(3)
        lib().orc_trilinear(self.h, _ptr(x), _ptr(out))
        return out

    def pose(self, p, t):
        o = np.zeros(3)
        v = np.zeros(3)
        lib().orc_pose(self.h, int(t), int(p), _ptr(o), _ptr(v))
        return o, v


def ibb_link(q, i, qf, rho_f, uf, uff, uw, Gp):
    """Eqs. 23-25 for one link: G_i(x_f, t + 1) with i the direction away from the wall."""
    return float(lib().orc_ibb_link(int(q), int(i), float(qf), float(rho_f), _d3(uf), _d3(uff), _d3(uw), float(Gp)))
