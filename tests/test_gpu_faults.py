"""Failure detection without any GPU fault: faults are injected on the host.

- A population poisoned with NaN in a checkpoint file (on the host, before upload) propagates
  through the LBM into the velocity field; the walker pass counts the non-finite velocities and
  rwmi_sync reports RWMI_E_NONFINITE.
- A served request cancelled while it runs is closed between chunks; the other requests finish
  with the results they have when run alone.
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
