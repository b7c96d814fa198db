"""Binning without allocation: rwmi_bin_walkers_noalloc against the library's own binning.

Some callers cannot allocate device memory: an external memory manager owns all of it, or the
call sits in a captured or real-time pipeline where cudaMalloc is not allowed. For them the
library bins (and cell-sorts) walkers with scratch held in a fixed array compiled into the
library. This file checks, through the C ABI, that two calls in a row give exactly the counts of
rwmi_concentration, and that the sorted copy is the same walkers grouped by cell. It is named so
that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _cells(pos, dims, wall_mask):
    """Cell of each walker: floor, wrapped on periodic axes, clamped on walled ones."""
    c = []
    for a in range(3):
        i = np.floor(pos[:, a]).astype(np.int64)
        i = np.clip(i, 0, dims[a] - 1) if (wall_mask >> a) & 1 else np.mod(i, dims[a])
        c.append(i)
    return (c[2] * dims[1] + c[1]) * dims[0] + c[0]


def test_noalloc_binning_matches_the_library_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation, bin_walkers_noalloc, load

    load()
    w = I.ragged(n_walkers=20000)
    sim = Simulation.from_workload(w)
    n_cells = int(np.prod(w.dims))
    stream = torch.cuda.Stream()
    for call in range(2):
        sim.step(7)
        pos, ids, _ = sim.walkers(with_x0=False)
        expect = sim.concentration()
        pos4 = np.concatenate([pos, ids.astype(np.uint32).view(np.float32)[:, None]], axis=1)
        posd = torch.from_numpy(np.ascontiguousarray(pos4)).cuda()
        # must be overwritten; on the second call it starts 4 bytes into its storage, so the scan
        # takes its word-by-word path instead of 16-byte accesses
        counts = torch.full((n_cells + call,), 7, dtype=torch.int32, device="cuda")[call:]
        out = torch.full_like(posd, -1.0)
        with torch.cuda.stream(stream):
            bin_walkers_noalloc(w.dims, w.wall_mask, posd, counts, out, stream=stream)
        stream.synchronize()
        got = counts.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, expect), f"call {call}: counts differ"
        s = out.cpu().numpy()
        sid = s[:, 3].view(np.uint32)
        assert np.array_equal(np.sort(sid), np.sort(ids.astype(np.uint32)))
        cells = _cells(s[:, :3], w.dims, w.wall_mask)
        assert np.all(np.diff(cells) >= 0), "not grouped by ascending cell"
        assert np.array_equal(np.bincount(cells, minlength=n_cells), expect)
        # each walker keeps its own position
        order = np.argsort(ids)
        assert np.array_equal(s[np.argsort(sid)][:, :3], pos[order])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300.rwmi import RwmiError, bin_walkers_noalloc

    pos = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    counts = torch.zeros(128 ** 3, dtype=torch.int32, device="cuda")   # a valid buffer: the library refuses
    with pytest.raises(RwmiError, match="1048576"):
        bin_walkers_noalloc((128, 128, 128), 0, pos, counts)   # 2^21 cells > 2^20


def _cell_of(v, n, walled):
    """Exact cell of one binary32 coordinate: Python integers, no rounding."""
    import math
    v = float(np.float32(v))
    if math.isnan(v):
        return 0
    if math.isinf(v):
        return (n - 1 if v > 0 else 0) if walled else 0
    i = math.floor(v)
    return min(max(i, 0), n - 1) if walled else i % n


def test_noalloc_counts_every_walker_inside_the_box_for_any_position():
    """Unwrapped coordinates far outside the box (+-1e9, +-1e30, 2^40 + 4, where a binary32
    quotient by the box size is off by many periods) and NaN or infinite ones: every walker is
    counted in a cell of the box (its exact residue on a periodic axis, the clamped end on a
    walled one; NaN and infinities in cell 0 of a periodic axis), so the counts sum to n and the
    sorted copy holds every walker."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300.rwmi import bin_walkers_noalloc, load

    load()
    dims, wall_mask = (7, 5, 6), 4            # z walled, x and y periodic
    vals = [0.5, 3.25, -0.75, 1e9, -1e9, 1e30, -1e30, 123456789.0, 2.0 ** 40 + 4, np.inf, -np.inf, np.nan]
    rng = np.random.default_rng(5)
    pos = []
    for a in range(3):
        for v in vals:
            p = rng.uniform(0.0, 5.0, 3)
            p[a] = v
            pos.append(p)
    pos = np.array(pos, np.float32)
    n = len(pos)
    want = np.zeros(np.prod(dims), np.int64)
    for p in pos:
        c = [_cell_of(p[a], dims[a], (wall_mask >> a) & 1) for a in range(3)]
        want[(c[2] * dims[1] + c[1]) * dims[0] + c[0]] += 1
    pos4 = np.concatenate([pos, np.arange(n, dtype=np.uint32).view(np.float32)[:, None]], axis=1)
    posd = torch.from_numpy(np.ascontiguousarray(pos4)).cuda()
    counts = torch.full((int(np.prod(dims)),), 9, dtype=torch.int32, device="cuda")
    out = torch.zeros_like(posd)
    bin_walkers_noalloc(dims, wall_mask, posd, counts, out)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint32)
    assert got.sum() == n
    assert np.array_equal(got, want)
    assert np.array_equal(np.sort(out.cpu().numpy()[:, 3].view(np.uint32)), np.arange(n))


def test_noalloc_binding_refuses_bad_buffers():
    """The Python binding checks device, dtype, contiguity, sizes and overlap before the call."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05007_gb300.rwmi import bin_walkers_noalloc

    pos = torch.zeros((16, 4), dtype=torch.float32, device="cuda")
    counts = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError, match="counts holds"):
        bin_walkers_noalloc((4, 4, 5), 0, pos, counts)                      # 80 cells > 64
    with pytest.raises(ValueError, match="overlap"):
        bin_walkers_noalloc((4, 4, 4), 0, pos, counts, pos)
    with pytest.raises(ValueError, match="current CUDA device"):
        bin_walkers_noalloc((4, 4, 4), 0, pos.cpu(), counts)
    with pytest.raises(ValueError, match="4 floats"):
        bin_walkers_noalloc((4, 4, 4), 0, pos.reshape(-1)[:30], counts)
    with pytest.raises(ValueError, match="dtype"):
        bin_walkers_noalloc((4, 4, 4), 0, pos, counts.to(torch.int64))
