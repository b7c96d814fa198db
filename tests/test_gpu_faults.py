"""Failure detection without any GPU fault: faults are injected on the host.

- A population poisoned with NaN in a checkpoint file (on the host, before upload) propagates
  through the LBM into the velocity field; the walker pass counts the non-finite velocities and
  rwmi_sync reports RWMI_E_NONFINITE.
- A served request cancelled while it runs is closed between chunks; the other requests finish
  with the results they have when run alone.
- Each device allocation in turn is made to fail on the host (rwmi_inject_alloc_failure, which
  never reaches the CUDA allocator): the call reports RWMI_E_OOM, the context is fenced (later
  calls return RWMI_E_STATE and keep the first message), it is destroyed as far as it was
  built, and a clean run afterwards gives the same results bit for bit.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_poisoned_population_is_reported_nonfinite(tmp_path):
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import RwmiError, Simulation
    w = I.ragged(n_walkers=3000)
    path = os.fspath(tmp_path / "ckpt.bin")
    with Simulation.from_workload(w) as s:
        s.step(4)
        assert s.sync() >= 0
        s.save(path)
    raw = bytearray(open(path, "rb").read())
    header = 10 * 8
    n_cells = int(np.prod(w.dims))
    rest = np.frombuffer(raw, dtype=np.float32, count=n_cells, offset=header).copy()
    rest[:] = np.nan                       # direction 0 of every cell (binary32 shifted storage)
    raw[header:header + 4 * n_cells] = rest.tobytes()
    open(path, "wb").write(bytes(raw))
    with Simulation.from_workload(w) as s:
        s.load(path)
        s.step(2)
        with pytest.raises(RwmiError, match="NONFINITE"):
            s.sync()


def test_cancelled_request_leaves_the_others_intact():
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation
    from paper_2308_05007_gb300.serve import Server, gpu_backend

    reqs = I.served(n_requests=4, rate=500.0, seed=12, edge=(24, 40), walkers=(1000, 5000),
                    steps=(64, 160), storage=(1,))

    def collect(sim, w):
        return dict(c=sim.concentration(), u=sim.velocity())

    srv = Server(gpu_backend(collect), budget_bytes=1 << 34, max_active=4, chunk_cell_updates=24 ** 3 * 16)
    victim = reqs[1].rid

    def on_event(kind, rec):
        if kind == "admit" and rec.rid == victim:
            srv.cancel(victim)

    rep = srv.run(reqs, on_event=on_event)
    by_id = {r.rid: r for r in rep.records}
    assert by_id[victim].cancelled and by_id[victim].result is None
    for r in reqs:
        if r.rid == victim:
            continue
        rec = by_id[r.rid]
        assert not rec.cancelled
        with Simulation.from_workload(r.workload) as s:
            s.step(r.workload.steps)
            alone = collect(s, r.workload)
        assert np.array_equal(alone["c"], rec.result["c"])
        assert np.array_equal(alone["u"], rec.result["u"])


def _run_all(w, keep):
    """Create, configure, particles (and free DEM), walkers, 4 steps and the outputs, one call
    at a time; the context goes into `keep` as soon as it exists."""
    from paper_2308_05007_gb300.rwmi import Simulation
    s = Simulation(w.dims, w.tau, w.D, w.seed, q=w.q, storage=w.storage, wall_mask=w.wall_mask,
                   body_force=w.body_force, force_period=w.force_period, rho0=w.rho0,
                   init_velocity=w.init_velocity, sort_interval=4, moment_interval=4,
                   coupling=getattr(w, "coupling", 0))
    keep.append(s)
    s.set_metaballs(w.metaballs)
    if getattr(w, "dem", None) is not None:
        s.set_dem(w.dem)
    s.seed_walkers(w.n_walkers, *w.walker_box)
    s.step(4)
    s.sync()
    pos, x0 = s.walkers_by_id()     # by walker id: the order within a cell is not fixed
    return dict(c=s.concentration(), u=s.velocity(), f=s.populations(), x=pos, x0=x0)


@pytest.mark.parametrize("kind", ["psm", "ibb_dem"])
def test_every_allocation_failure_is_reported_and_fences_the_context(kind):
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300 import rwmi as R
    if kind == "psm":
        w = I.ragged(n_walkers=500)
    else:
        w = I.with_(I.dem_box(n_particles=3, n_walkers=500), coupling=1)
    R.inject_alloc_failure(-1)
    keep = []
    n0 = R.alloc_count()
    ref = _run_all(w, keep)
    n_alloc = R.alloc_count() - n0
    keep.pop().close()
    assert n_alloc > 20
    fenced = 0
    for k in range(n_alloc):
        keep = []
        R.inject_alloc_failure(k)
        try:
            with pytest.raises(R.RwmiError) as e:
                _run_all(w, keep)
        finally:
            R.inject_alloc_failure(-1)
        assert e.value.status == -2, (k, str(e.value))
        if keep:
            s = keep[0]
            msg = s._L.rwmi_last_error(s._h).decode()
            assert "out of memory" in msg, msg
            for call in (lambda: s.step(1), s.sync, s.velocity):
                with pytest.raises(R.RwmiError) as e2:
                    call()
                assert e2.value.status == -6, (k, str(e2.value))
            assert s._L.rwmi_last_error(s._h).decode() == msg
            s.close()
            fenced += 1
    assert fenced > 0
    again = []
    res = _run_all(w, again)
    again.pop().close()
    for key in ref:
        assert np.array_equal(ref[key], res[key]), key
