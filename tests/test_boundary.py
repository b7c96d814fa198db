"""The C-ABI library builds for sm_103a, loads, and exports exactly what include/rwmi.h declares
(no compute calls: this runs on machines without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rwmi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"RWMI_API[^;{(]*?\b(rwmi_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2308_05007_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rwmi_create", "rwmi_set_metaballs", "rwmi_step", "rwmi_concentration",
                     "rwmi_walker_moments", "rwmi_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(rwmi_\w+)\b", out))
    assert set(_declared()) <= exported, set(_declared()) - exported
    # nothing else leaks out of the C ABI
    assert exported == set(_declared())


def test_every_translation_unit_builds_for_sm_103a_only():
    from paper_2308_05007_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    flags = " ".join(build.FLAGS + [f for v in build.SOURCE_FLAGS.values() for f in v])
    assert "gencode" not in flags and "-arch" not in flags
    csrc = sorted(f for f in os.listdir(build.CSRC) if f.endswith(".cu"))
    assert sorted(build.SOURCES) == csrc


def test_binding_loads_and_matches_header(lib_path):
    from paper_2308_05007_gb300 import rwmi
    L = rwmi.load()
    assert set(rwmi.EXPORTED) == set(_declared())
    for name in rwmi.EXPORTED:
        assert hasattr(L, name)


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    """The product path has no fallback: a missing library is an error."""
    from paper_2308_05007_gb300 import build, rwmi
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rwmi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        rwmi.load()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2308_05007_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", text).lower() or f == "inputs.py", f


# ---- host-only entry points: argument checks and sizes, callable without a GPU ----
def _L(lib_path):
    from paper_2308_05007_gb300 import rwmi
    return rwmi, rwmi.load()


def test_invalid_create_arguments_are_refused_before_any_cuda_call(lib_path):
    import ctypes as C
    rwmi, L = _L(lib_path)
    h = C.c_void_p()
    for dims, tau, D in (((0, 4, 4), 0.8, 0.01), ((4, 4, 4), 0.5, 0.01), ((4, 4, 4), float("nan"), 0.01),
                         ((4, 4, 4), 0.8, -1.0), ((4, 4, 4), 0.8, float("inf")), ((1 << 21, 1, 1), 0.8, 0.0),
                         ((1 << 11, 1 << 11, 1 << 10), 0.8, 0.0)):
        d = (C.c_int32 * 3)(*dims)
        assert L.rwmi_create(C.byref(h), d, tau, D, C.c_uint64(0)) == -1, (dims, tau, D)
        assert h.value is None
    assert L.rwmi_create(None, (C.c_int32 * 3)(4, 4, 4), 0.8, 0.0, C.c_uint64(0)) == -1


def test_null_handles_are_refused(lib_path):
    import ctypes as C
    rwmi, L = _L(lib_path)
    assert L.rwmi_step(None, 1) == -1
    assert L.rwmi_sync(None) == -1
    assert L.rwmi_configure(None, None) == -1
    assert L.rwmi_concentration(None, None) == -1
    assert L.rwmi_launch_count(None) == 0
    assert isinstance(L.rwmi_last_error(None), bytes)
    L.rwmi_destroy(None)
    L.rwmi_batch_destroy(None)
    out = C.c_void_p()
    assert L.rwmi_batch_create(C.byref(out), None, 0) == -1
    assert L.rwmi_batch_step(None, 16) == -1
    assert L.rwmi_batch_set_mode(None, 0) == -1
    assert L.rwmi_batch_set_tiles(None, None) == -1
    assert L.rwmi_batch_get_tiles(None, None) == -1
    assert L.rwmi_batch_autotune(None, 16, None) == -1
    assert L.rwmi_batch_launch_count(None) == 0
    n = C.c_int32()
    assert L.rwmi_force_series(None, None, 0, C.byref(n)) == -1


def test_defaults_are_the_documented_ones(lib_path):
    import ctypes as C
    rwmi, L = _L(lib_path)
    cfg = rwmi.Config()
    L.rwmi_config_defaults(C.byref(cfg))
    assert (cfg.q, cfg.storage, cfg.wall_mask, cfg.rho0, cfg.sort_interval, cfg.moment_interval,
            cfg.use_graphs, cfg.lbm_block, cfg.overlap, cfg.coupling,
            cfg.lbm_staging, cfg.force_interval) == (19, 1, 0, 1.0, 16, 0, 1, 128, 2, 0, 0, 0)
    assert list(cfg.body_force) == [0.0] * 3 and cfg.force_period == 0.0
    dem = rwmi.DemConfig()
    L.rwmi_dem_defaults(C.byref(dem))
    assert (dem.kn, dem.eta_n, dem.kt, dem.eta_t, dem.mu_s, dem.substeps, dem.hydro) == (200.0, 0, 0, 0, 0, 10, 1)
    assert list(dem.gravity) == [0.0] * 3


def test_footprint_follows_the_storage_layout(lib_path):
    """Device bytes of a context: the two population buffers hold q x (cells + 1 rounded up to
    64) values of the storage's width; everything else is independent of q and the storage."""
    rwmi, _ = _L(lib_path)
    dims, pad = (40, 36, 26), (40 * 36 * 26 + 64) // 64 * 64
    base = dict(n_walkers=12345, n_particles=5, n_centers=17)
    fp = {(q, st): rwmi.footprint(dims, q, st, **base) for q in (15, 19) for st in (0, 1, 2, 3)}
    width = {0: 4, 1: 4, 2: 2, 3: 8}
    for q in (15, 19):
        for st in (1, 2, 3):
            assert fp[q, st] - fp[q, 0] == 2 * q * pad * (width[st] - 4)
    for st in (0, 1, 2, 3):
        assert fp[19, st] - fp[15, st] == 2 * 4 * pad * width[st]
    more = rwmi.footprint(dims, 15, 1, n_walkers=2 * 12345, n_particles=5, n_centers=17)
    assert more > fp[15, 1]
    for bad in (dict(q=17), dict(storage=4), dict(n_walkers=-1)):
        kw = dict(q=15, storage=1, **base)
        kw.update(bad)
        with pytest.raises(rwmi.RwmiError):
            rwmi.footprint(dims, kw["q"], kw["storage"], kw["n_walkers"], kw["n_particles"], kw["n_centers"])
    with pytest.raises(rwmi.RwmiError):
        rwmi.footprint((0, 4, 4), 15, 1, 0, 0, 0)


def test_allocation_failure_injection_is_armed_and_disarmed_on_the_host(lib_path):
    rwmi, _ = _L(lib_path)
    n = rwmi.alloc_count()
    assert rwmi.inject_alloc_failure(5) == n
    assert rwmi.inject_alloc_failure(-1) == n     # no allocation was made in between
    assert rwmi.alloc_count() == n
