"""Thin ctypes binding of librwmi.so (include/rwmi.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module converts numpy/torch
arrays to pointers and status codes to exceptions. If the library is missing it raises -- there
is no CPU path.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

RWMI_OK, RWMI_W_BISECT, RWMI_W_SEED, RWMI_BUSY = 0, 1, 2, 3
STATUS_NAMES = {0: "RWMI_OK", 1: "RWMI_W_BISECT", 2: "RWMI_W_SEED", 3: "RWMI_BUSY", -1: "RWMI_E_INVALID", -2: "RWMI_E_OOM",
                -3: "RWMI_E_CUDA", -4: "RWMI_E_NONFINITE", -5: "RWMI_E_TIMEOUT", -6: "RWMI_E_STATE"}
STORE_FP32, STORE_FP32_SHIFT, STORE_FP16_SHIFT, STORE_FP64_SHIFT = 0, 1, 2, 3

EXPORTED = ["rwmi_config_defaults", "rwmi_create", "rwmi_configure", "rwmi_set_stream",
            "rwmi_set_metaballs", "rwmi_seed_walkers", "rwmi_set_walkers", "rwmi_step", "rwmi_step_timed",
            "rwmi_autotune", "rwmi_query", "rwmi_footprint", "rwmi_sync",
            "rwmi_time", "rwmi_info", "rwmi_concentration", "rwmi_walker_moments", "rwmi_moment_series",
            "rwmi_velocity", "rwmi_density", "rwmi_populations", "rwmi_lattice", "rwmi_solid", "rwmi_nodes",
            "rwmi_mass_momentum", "rwmi_particle_forces", "rwmi_force_series", "rwmi_walkers", "rwmi_counters",
            "rwmi_save",
            "rwmi_load", "rwmi_brick_stats", "rwmi_bin_walkers_noalloc", "rwmi_last_error",
            "rwmi_launch_count", "rwmi_destroy", "rwmi_batch_create", "rwmi_batch_step", "rwmi_batch_sync",
            "rwmi_batch_last_error", "rwmi_batch_destroy", "rwmi_dem_defaults", "rwmi_set_dem",
            "rwmi_particle_state", "rwmi_set_particle_state", "rwmi_particle_mass",
            "rwmi_inject_alloc_failure", "rwmi_alloc_count", "rwmi_inject_wait_timeout", "rwmi_batch_set_mode",
            "rwmi_batch_get_tiles",
            "rwmi_batch_set_tiles", "rwmi_batch_autotune", "rwmi_batch_launch_count"]
BATCH_AUTO, BATCH_BRANCHES, BATCH_FUSED = 0, 1, 2


class RwmiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class RwmiWarning(RuntimeWarning):
    pass


class Config(C.Structure):
    _fields_ = [("q", C.c_int32), ("storage", C.c_int32), ("wall_mask", C.c_uint32),
                ("body_force", C.c_double * 3), ("force_period", C.c_double), ("rho0", C.c_double),
                ("init_velocity", C.c_double * 3), ("sort_interval", C.c_int32),
                ("moment_interval", C.c_int32), ("use_graphs", C.c_int32), ("lbm_block", C.c_int32),
                ("overlap", C.c_int32), ("coupling", C.c_int32), ("lbm_staging", C.c_int32),
                ("force_interval", C.c_int32)]


class BatchTiles(C.Structure):
    """rwmi_batch_tiles: the work split of a fused batch's launches."""
    _fields_ = [("lbm_block", C.c_int32), ("walker_chunks_per_block", C.c_int32),
                ("resolve_walkers_per_block", C.c_int32), ("raster_bricks_per_block", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class DemConfig(C.Structure):
    _fields_ = [("kn", C.c_double), ("eta_n", C.c_double), ("kt", C.c_double), ("eta_t", C.c_double),
                ("mu_s", C.c_double), ("gravity", C.c_double * 3), ("substeps", C.c_int32),
                ("hydro", C.c_int32)]


_lib = None
_live = weakref.WeakSet()


@atexit.register
def _close_all():
    """Destroy every live context before interpreter teardown (the CUDA runtime must still exist)."""
    for sim in list(_live):
        try:
            sim.close()
        except Exception:
            pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load librwmi.so. Raises if it is not built (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is not built; run __graft_entry__.build() (needs nvcc)")
        _build.build()
    L = C.CDLL(_build.LIB)
    P, vp = C.c_void_p, C.c_void_p
    L.rwmi_config_defaults.argtypes = [C.POINTER(Config)]
    L.rwmi_config_defaults.restype = None
    L.rwmi_create.argtypes = [C.POINTER(P), C.POINTER(C.c_int32), C.c_double, C.c_double, C.c_uint64]
    L.rwmi_configure.argtypes = [P, C.POINTER(Config)]
    L.rwmi_set_stream.argtypes = [P, vp]
    L.rwmi_set_metaballs.argtypes = [P, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rwmi_seed_walkers.argtypes = [P, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.rwmi_set_walkers.argtypes = [P, C.c_int64, vp]
    L.rwmi_step.argtypes = [P, C.c_int32]
    L.rwmi_step_timed.argtypes = [P, C.c_int32, vp]
    L.rwmi_autotune.argtypes = [P, C.POINTER(C.c_int32)]
    L.rwmi_query.argtypes = [P]
    L.rwmi_footprint.argtypes = [C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                 C.POINTER(C.c_uint64)]
    L.rwmi_sync.argtypes = [P]
    L.rwmi_time.argtypes = [P, C.POINTER(C.c_int64)]
    L.rwmi_info.argtypes = [P, vp]
    for name in ("rwmi_concentration", "rwmi_walker_moments", "rwmi_velocity", "rwmi_density",
                 "rwmi_populations", "rwmi_mass_momentum", "rwmi_particle_forces", "rwmi_counters"):
        getattr(L, name).argtypes = [P, vp]
    L.rwmi_moment_series.argtypes = [P, vp, C.c_int32, C.POINTER(C.c_int32)]
    L.rwmi_force_series.argtypes = [P, vp, C.c_int32, C.POINTER(C.c_int32)]
    L.rwmi_lattice.argtypes = [P, vp, vp, C.POINTER(C.c_int32)]
    L.rwmi_solid.argtypes = [P, vp, vp]
    L.rwmi_nodes.argtypes = [P, vp]
    L.rwmi_walkers.argtypes = [P, vp, vp]
    L.rwmi_brick_stats.argtypes = [P, vp]
    L.rwmi_bin_walkers_noalloc.argtypes = [C.POINTER(C.c_int32), C.c_uint32, vp, C.c_int64, vp, vp, vp]
    L.rwmi_save.argtypes = [P, C.c_char_p]
    L.rwmi_load.argtypes = [P, C.c_char_p]
    L.rwmi_last_error.argtypes = [P]
    L.rwmi_last_error.restype = C.c_char_p
    L.rwmi_launch_count.argtypes = [P]
    L.rwmi_launch_count.restype = C.c_int64
    L.rwmi_destroy.argtypes = [P]
    L.rwmi_destroy.restype = None
    L.rwmi_batch_create.argtypes = [C.POINTER(P), C.POINTER(P), C.c_int32]
    L.rwmi_batch_step.argtypes = [P, C.c_int32]
    L.rwmi_batch_sync.argtypes = [P]
    L.rwmi_batch_last_error.argtypes = [P]
    L.rwmi_batch_last_error.restype = C.c_char_p
    L.rwmi_batch_destroy.argtypes = [P]
    L.rwmi_batch_destroy.restype = None
    L.rwmi_dem_defaults.argtypes = [C.POINTER(DemConfig)]
    L.rwmi_dem_defaults.restype = None
    L.rwmi_set_dem.argtypes = [P, C.POINTER(DemConfig), vp, vp, vp, vp]
    L.rwmi_particle_state.argtypes = [P, vp]
    L.rwmi_particle_mass.argtypes = [P, vp]
    L.rwmi_set_particle_state.argtypes = [P, vp]
    L.rwmi_inject_alloc_failure.argtypes = [C.c_int64]
    L.rwmi_inject_alloc_failure.restype = C.c_int64
    L.rwmi_alloc_count.argtypes = []
    L.rwmi_alloc_count.restype = C.c_int64
    L.rwmi_inject_wait_timeout.argtypes = [C.c_int32]
    L.rwmi_inject_wait_timeout.restype = C.c_int32
    L.rwmi_batch_set_mode.argtypes = [P, C.c_int32]
    L.rwmi_batch_get_tiles.argtypes = [P, C.POINTER(BatchTiles)]
    L.rwmi_batch_set_tiles.argtypes = [P, C.POINTER(BatchTiles)]
    L.rwmi_batch_autotune.argtypes = [P, C.c_int32, C.POINTER(BatchTiles)]
    L.rwmi_batch_launch_count.argtypes = [P]
    L.rwmi_batch_launch_count.restype = C.c_int64
    for name in EXPORTED:
        fn = getattr(L, name)
        if name not in ("rwmi_config_defaults", "rwmi_last_error", "rwmi_launch_count", "rwmi_destroy",
                        "rwmi_batch_last_error", "rwmi_batch_destroy", "rwmi_dem_defaults",
                        "rwmi_inject_alloc_failure", "rwmi_alloc_count", "rwmi_batch_launch_count",
                        "rwmi_inject_wait_timeout"):
            fn.restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    """Pointer of a numpy array or a torch tensor (host or CUDA)."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _d3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def footprint(dims, q, storage, n_walkers, n_particles, n_centers) -> int:
    """Device bytes a context of these sizes needs (rwmi_footprint)."""
    L = load()
    d = (C.c_int32 * 3)(*[int(x) for x in dims])
    out = C.c_uint64()
    st = L.rwmi_footprint(d, int(q), int(storage), int(n_walkers), int(n_particles), int(n_centers), C.byref(out))
    if st != 0:
        raise RwmiError(st, "rwmi_footprint: bad sizes")
    return int(out.value)


def inject_alloc_failure(after: int) -> int:
    """rwmi_inject_alloc_failure: the device allocation `after` allocations from now reports
    RWMI_E_OOM without reaching the allocator (after < 0 disarms). Returns the count so far."""
    return int(load().rwmi_inject_alloc_failure(int(after)))


def inject_wait_timeout(launches: int) -> int:
    """rwmi_inject_wait_timeout: the next `launches` TMA-staged LBM updates let one bounded wait
    expire (rwmi_sync then reports RWMI_E_TIMEOUT); <= 0 disarms. Returns the previous count."""
    return int(load().rwmi_inject_wait_timeout(int(launches)))


def alloc_count() -> int:
    """rwmi_alloc_count: device allocations made (or refused by injection) in this process."""
    return int(load().rwmi_alloc_count())


def bin_walkers_noalloc(dims, wall_mask, pos, counts, pos_sorted=None, stream=None):
    """rwmi_bin_walkers_noalloc: walkers per cell (and, optionally, the walkers grouped by cell)
    for callers that cannot allocate device memory. pos, counts, pos_sorted are CUDA tensors
    (float32 [n, 4], uint32/int32 [cells], float32 [n, 4]); asynchronous on `stream`."""
    import torch
    L = load()
    dims = tuple(int(x) for x in dims)
    if len(dims) != 3 or min(dims) < 1:
        raise ValueError("dims must be three positive sizes")
    n_cells = dims[0] * dims[1] * dims[2]
    dev = torch.device("cuda", torch.cuda.current_device())
    int32_types = {torch.int32} | ({torch.uint32} if hasattr(torch, "uint32") else set())

    def _check(t, name, dtypes, min_numel):
        if not isinstance(t, torch.Tensor) or t.device != dev:
            raise ValueError(f"{name} must be a tensor on the current CUDA device {dev}")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} has dtype {t.dtype}, expected one of {sorted(map(str, dtypes))}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < min_numel:
            raise ValueError(f"{name} holds {t.numel()} elements, needs {min_numel}")

    _check(pos, "pos", {torch.float32}, 0)
    if pos.numel() % 4:
        raise ValueError("pos must hold 4 floats per walker")
    _check(counts, "counts", int32_types, n_cells)
    if pos_sorted is not None:
        _check(pos_sorted, "pos_sorted", {torch.float32}, pos.numel())
        a0, a1 = pos.data_ptr(), pos.data_ptr() + 4 * pos.numel()
        b0, b1 = pos_sorted.data_ptr(), pos_sorted.data_ptr() + 4 * pos.numel()
        if pos.numel() and a0 < b1 and b0 < a1:
            raise ValueError("pos_sorted must not overlap pos")
    d = (C.c_int32 * 3)(*dims)
    n = pos.numel() // 4
    handle = None
    if stream is not None:
        handle = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    st = L.rwmi_bin_walkers_noalloc(d, int(wall_mask), _ptr(pos), n,
                                    _ptr(pos_sorted) if pos_sorted is not None else None, _ptr(counts), handle)
    if st != 0:
        raise RwmiError(st, L.rwmi_last_error(None).decode(errors="replace"))


class Simulation:
    """One GPU simulation context (librwmi.so). Outputs are numpy arrays unless a torch tensor
    (host or CUDA, contiguous, right dtype and size) is passed as ``out``."""

    def __init__(self, dims, tau, D, seed=0, q=19, storage=STORE_FP32_SHIFT, wall_mask=0,
                 body_force=(0.0, 0.0, 0.0), force_period=0.0, rho0=1.0, init_velocity=(0.0, 0.0, 0.0),
                 sort_interval=16, moment_interval=0, use_graphs=True, stream=None, lbm_block=128,
                 overlap=2, coupling=0, lbm_staging=0, force_interval=0):
        L = load()
        self._L = L
        self._h = C.c_void_p()
        d = (C.c_int32 * 3)(*[int(x) for x in dims])
        st = L.rwmi_create(C.byref(self._h), d, float(tau), float(D), C.c_uint64(int(seed) & (2**64 - 1)))
        if st != 0:
            raise RwmiError(st, "rwmi_create failed")
        self.dims = tuple(int(x) for x in dims)
        self.n_cells = self.dims[0] * self.dims[1] * self.dims[2]
        cfg = Config()
        L.rwmi_config_defaults(C.byref(cfg))
        cfg.q, cfg.storage, cfg.wall_mask = int(q), int(storage), int(wall_mask)
        for a in range(3):
            cfg.body_force[a] = float(body_force[a])
            cfg.init_velocity[a] = float(init_velocity[a])
        cfg.force_period, cfg.rho0 = float(force_period), float(rho0)
        cfg.sort_interval, cfg.moment_interval = int(sort_interval), int(moment_interval)
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.lbm_block = int(lbm_block)
        cfg.overlap = int(overlap)
        cfg.coupling = int(coupling)
        cfg.lbm_staging = int(lbm_staging)
        cfg.force_interval = int(force_interval)
        try:
            self._check(L.rwmi_configure(self._h, C.byref(cfg)))
        except RwmiError:
            self.close()
            raise
        self.q = int(q)
        _live.add(self)
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def from_workload(cls, w, seed_walkers=True, **overrides):
        kw = dict(q=w.q, storage=w.storage, wall_mask=w.wall_mask, body_force=w.body_force,
                  force_period=w.force_period, rho0=w.rho0, init_velocity=w.init_velocity,
                  sort_interval=w.sort_interval, moment_interval=w.moment_interval,
                  coupling=getattr(w, "coupling", 0))
        kw.update(overrides)
        s = cls(w.dims, w.tau, w.D, w.seed, **kw)
        if w.metaballs is not None and w.metaballs.n_particles > 0:
            s.set_metaballs(w.metaballs)
            if getattr(w, "dem", None) is not None:
                s.set_dem(w.dem)
        if seed_walkers and w.n_walkers:
            if w.walker_positions is not None:
                s.set_walkers(w.walker_positions)
            else:
                s.seed_walkers(w.n_walkers, *w.walker_box)
        return s

    # ---- plumbing ----
    def _check(self, st):
        if st < 0:
            raise RwmiError(st, self._L.rwmi_last_error(self._h).decode(errors="replace"))
        return st

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.rwmi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._check(self._L.rwmi_set_stream(self._h, C.c_void_p(handle)))

    # ---- setup ----
    def set_metaballs(self, mb):
        keep = dict(
            coff=np.ascontiguousarray(mb.center_offsets, np.int32),
            cb=np.ascontiguousarray(mb.centers_body, np.float32).reshape(-1),
            k=np.ascontiguousarray(mb.k, np.float32),
            org=np.ascontiguousarray(mb.origin, np.float64).reshape(-1),
            amp=np.ascontiguousarray(mb.amplitude, np.float64).reshape(-1),
            per=np.ascontiguousarray(mb.period, np.float64),
            pha=np.ascontiguousarray(mb.phase, np.float64),
            omg=np.ascontiguousarray(mb.omega, np.float64).reshape(-1))
        P = len(keep["coff"]) - 1
        self._check(self._L.rwmi_set_metaballs(self._h, P, _ptr(keep["coff"]), _ptr(keep["cb"]), _ptr(keep["k"]),
                                               _ptr(keep["org"]), _ptr(keep["amp"]), _ptr(keep["per"]),
                                               _ptr(keep["pha"]), _ptr(keep["omg"])))

    def set_dem(self, dem):
        """Free DEM (Eqs. 4-11) from the current time; `dem` has the fields of inputs.Dem."""
        cfg = DemConfig()
        self._L.rwmi_dem_defaults(C.byref(cfg))
        cfg.kn, cfg.eta_n, cfg.kt, cfg.eta_t, cfg.mu_s = (float(dem.kn), float(dem.eta_n), float(dem.kt),
                                                          float(dem.eta_t), float(dem.mu_s))
        for a in range(3):
            cfg.gravity[a] = float(dem.gravity[a])
        cfg.substeps, cfg.hydro = int(dem.substeps), int(dem.hydro)
        P = self.n_particles
        keep = dict(rho=np.ascontiguousarray(np.broadcast_to(dem.density, (P,)), np.float64),
                    Rs=np.ascontiguousarray(dem.sphere_radius, np.float64).reshape(P),
                    v=None if dem.velocity is None else np.ascontiguousarray(dem.velocity, np.float64).reshape(3 * P),
                    w=None if dem.spin is None else np.ascontiguousarray(dem.spin, np.float64).reshape(3 * P))
        self._check(self._L.rwmi_set_dem(self._h, C.byref(cfg), _ptr(keep["rho"]), _ptr(keep["Rs"]),
                                         None if keep["v"] is None else _ptr(keep["v"]),
                                         None if keep["w"] is None else _ptr(keep["w"])))

    def particle_mass(self):
        """[P, 10]: mass, centre of mass (given body frame), inertia about it (xx yy zz xy xz yz)."""
        out = np.zeros((self.n_particles, 10))
        self._check(self._L.rwmi_particle_mass(self._h, _ptr(out)))
        return out

    def particle_state(self, out=None):
        """Free-DEM state [P, 13]: origin (unwrapped), quaternion (w, x, y, z), velocity, spin."""
        out = self._out(out, (self.n_particles, 13), np.float64)
        self._check(self._L.rwmi_particle_state(self._h, _ptr(out)))
        return out

    def set_particle_state(self, st):
        st = np.ascontiguousarray(st, np.float64).reshape(self.n_particles, 13)
        self._check(self._L.rwmi_set_particle_state(self._h, _ptr(st)))

    def seed_walkers(self, n, lo, hi):
        st = self._check(self._L.rwmi_seed_walkers(self._h, int(n), _d3(lo), _d3(hi)))
        if st == RWMI_W_SEED:
            import warnings
            warnings.warn(self._L.rwmi_last_error(self._h).decode(), RwmiWarning)
        return st

    def set_walkers(self, pos):
        if hasattr(pos, "data_ptr"):
            n = pos.numel() // 3
            self._check(self._L.rwmi_set_walkers(self._h, n, _ptr(pos)))
        else:
            pos = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
            n = len(pos)
            self._check(self._L.rwmi_set_walkers(self._h, n, _ptr(pos)))

    # ---- stepping ----
    def step(self, n=1):
        self._check(self._L.rwmi_step(self._h, int(n)))

    PHASES = ("raster", "lbm", "pose_bricks", "walkers", "sort_bin", "moments")

    def step_timed(self, n=1) -> dict:
        """n eager steps with CUDA events around each phase; GPU milliseconds per phase (summed)."""
        out = np.zeros(len(self.PHASES))
        self._check(self._L.rwmi_step_timed(self._h, int(n), _ptr(out)))
        return dict(zip(self.PHASES, out.tolist()))

    def autotune(self) -> int:
        """Pick the LBM block size by timing (rwmi_autotune); returns it."""
        v = C.c_int32()
        self._check(self._L.rwmi_autotune(self._h, C.byref(v)))
        return int(v.value)

    def busy(self) -> bool:
        """True while GPU work of this context is in flight (rwmi_query, non-blocking)."""
        return self._check(self._L.rwmi_query(self._h)) == RWMI_BUSY

    def sync(self) -> int:
        return self._check(self._L.rwmi_sync(self._h))

    def info(self) -> dict:
        out = np.zeros(8, np.int64)
        self._check(self._L.rwmi_info(self._h, _ptr(out)))
        keys = ["nx", "ny", "nz", "q", "storage", "walkers", "particles", "t"]
        return dict(zip(keys, (int(v) for v in out)))

    @property
    def n_walkers(self) -> int:
        return self.info()["walkers"]

    @property
    def n_particles(self) -> int:
        return self.info()["particles"]

    @property
    def t(self) -> int:
        v = C.c_int64()
        self._check(self._L.rwmi_time(self._h, C.byref(v)))
        return int(v.value)

    @property
    def launch_count(self) -> int:
        return int(self._L.rwmi_launch_count(self._h))

    # ---- outputs ----
    def _out(self, out, shape, dtype):
        if out is None:
            out = np.zeros(shape, dtype)
        return out

    def concentration(self, out=None):
        out = self._out(out, self.n_cells, np.uint32)
        self._check(self._L.rwmi_concentration(self._h, _ptr(out)))
        return out

    def walker_moments(self, out=None):
        out = self._out(out, 13, np.float64)
        self._check(self._L.rwmi_walker_moments(self._h, _ptr(out)))
        return out

    def moment_series(self, max_rows=65536):
        out = np.zeros((max_rows, 14))
        n = C.c_int32()
        self._check(self._L.rwmi_moment_series(self._h, _ptr(out), max_rows, C.byref(n)))
        return out[: n.value]

    def velocity(self, out=None):
        out = self._out(out, (self.n_cells, 3), np.float32)
        self._check(self._L.rwmi_velocity(self._h, _ptr(out)))
        return out

    def density(self, out=None):
        out = self._out(out, self.n_cells, np.float32)
        self._check(self._L.rwmi_density(self._h, _ptr(out)))
        return out

    def populations(self, out=None):
        out = self._out(out, (self.q, self.n_cells), np.float64)
        self._check(self._L.rwmi_populations(self._h, _ptr(out)))
        return out

    def lattice(self):
        e = np.zeros((self.q, 3), np.int32)
        w = np.zeros(self.q)
        q = C.c_int32()
        self._check(self._L.rwmi_lattice(self._h, _ptr(e), _ptr(w), C.byref(q)))
        return e, w

    def solid(self):
        cnt = np.zeros(self.n_cells, np.int32)
        own = np.zeros(self.n_cells, np.int32)
        self._check(self._L.rwmi_solid(self._h, _ptr(cnt), _ptr(own)))
        return cnt, own

    def nodes(self):
        """IBB node classes of the current time: 0 fluid, 1 + particle index for solid nodes."""
        out = np.zeros(self.n_cells, np.int32)
        self._check(self._L.rwmi_nodes(self._h, _ptr(out)))
        return out

    def mass_momentum(self):
        out = np.zeros(4)
        self._check(self._L.rwmi_mass_momentum(self._h, _ptr(out)))
        return out

    def particle_forces(self):
        out = np.zeros((max(self.n_particles, 1), 6))
        self._check(self._L.rwmi_particle_forces(self._h, _ptr(out)))
        return out[: self.n_particles]

    def force_series(self, max_rows=4096):
        """rwmi_force_series: (steps [R] int64, forces [R, P, 6]) of the recorded rows, oldest
        first; forces[r, p] = (F_p, T_p) of the LBM update that completed steps[r]."""
        P = self.n_particles
        out = np.zeros((max(int(max_rows), 1), 1 + 6 * P))
        n = C.c_int32()
        self._check(self._L.rwmi_force_series(self._h, _ptr(out), int(max_rows), C.byref(n)))
        rows = out[: n.value]
        return rows[:, 0].astype(np.int64), rows[:, 1:].reshape(n.value, P, 6)

    def walkers(self, with_x0=True):
        """Returns (positions [N,3] float32, ids [N] int64, start positions [N,3] or None) in the
        library's current (cell-sorted) order."""
        n = self.n_walkers
        raw = np.zeros((n, 4), np.float32)
        x0 = np.zeros((n, 3), np.float32) if with_x0 else None
        self._check(self._L.rwmi_walkers(self._h, _ptr(raw), _ptr(x0) if with_x0 else None))
        ids = raw[:, 3].view(np.uint32).astype(np.int64)
        return raw[:, :3].copy(), ids, x0

    def walkers_by_id(self):
        pos, ids, x0 = self.walkers()
        order = np.argsort(ids)
        return pos[order], x0[order]

    def brick_stats(self) -> dict:
        out = np.zeros(4, np.int64)
        self._check(self._L.rwmi_brick_stats(self._h, _ptr(out)))
        return dict(zip(["raster_bricks", "walker_bricks", "max_candidates", "overflow_bricks"],
                        (int(v) for v in out)))

    def counters(self) -> dict:
        out = np.zeros(12, np.int64)
        self._check(self._L.rwmi_counters(self._h, _ptr(out)))
        keys = ["type_I", "type_II", "type_III", "type_IV", "bisect_fail", "refill_fail", "wall_fail",
                "seed_fail", "nonfinite", "long_steps", "resolved", "raster_queued"]
        return dict(zip(keys, (int(v) for v in out)))

    def save(self, path):
        self._check(self._L.rwmi_save(self._h, os.fsencode(path)))

    def load(self, path):
        self._check(self._L.rwmi_load(self._h, os.fsencode(path)))


class Batch:
    """rwmi_batch: many contexts advanced by one CUDA graph launch per chunk. Fused (the default
    where allowed: one launch per phase for all contexts) or as concurrent per-context branches
    (then each context should use its own stream for the branches to overlap)."""

    def __init__(self, sims, mode=None):
        self._L = load()
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s._h.value for s in self.sims])
        self._h = C.c_void_p()
        st = self._L.rwmi_batch_create(C.byref(self._h), arr, len(self.sims))
        if st != 0:
            raise RwmiError(st, "rwmi_batch_create: contexts must share the chunk length (<= 64)")
        if mode is not None:
            self.set_mode(mode)

    def set_mode(self, mode):
        """BATCH_AUTO, BATCH_BRANCHES or BATCH_FUSED (rwmi_batch_set_mode)."""
        self._check(self._L.rwmi_batch_set_mode(self._h, int(mode)))

    @property
    def tiles(self) -> dict:
        t = BatchTiles()
        self._check(self._L.rwmi_batch_get_tiles(self._h, C.byref(t)))
        return t.as_dict()

    def set_tiles(self, **kw):
        t = BatchTiles()
        self._check(self._L.rwmi_batch_get_tiles(self._h, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        self._check(self._L.rwmi_batch_set_tiles(self._h, C.byref(t)))

    def autotune(self, steps=16) -> dict:
        """rwmi_batch_autotune: picks the fused work split; advances every context."""
        t = BatchTiles()
        self._check(self._L.rwmi_batch_autotune(self._h, int(steps), C.byref(t)))
        return t.as_dict()

    @property
    def launch_count(self) -> int:
        return int(self._L.rwmi_batch_launch_count(self._h))

    def _check(self, st):
        if st < 0:
            raise RwmiError(st, self._L.rwmi_batch_last_error(self._h).decode(errors="replace"))
        return st

    def step(self, n):
        self._check(self._L.rwmi_batch_step(self._h, int(n)))

    def sync(self) -> int:
        """Waits for the batch; the worst status of its contexts (warnings are positive)."""
        return self._check(self._L.rwmi_batch_sync(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.rwmi_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
