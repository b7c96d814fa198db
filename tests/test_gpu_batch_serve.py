"""Batched and served forms on the GPU: the same results as contexts stepped alone, and as
the FP64 oracle.

- rwmi_batch: several ragged domains advanced by one graph launch per chunk -- fused (one launch
  per phase for all domains) or as per-context branches -- give, bit for bit, the populations,
  velocities, walker positions and counts of the same domains stepped one by one with
  rwmi_step, for any work split of the fused launches. FP64 sums (moments, mass) are reductions
  whose order of atomic adds may differ between runs, so they are compared to 1e-12 relative.
- A batched domain and a served request against the FP64 oracle, with the single-context
  trajectory tolerances.
- Block-size autotuning changes no per-cell result; rwmi_query and rwmi_footprint behave.
- The request loop: every request's result in a mix of concurrent requests equals its result
  alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _small_domains(n=3, seed=5):
    from paper_2308_05007_gb300 import inputs as I
    return I.batched(n_domains=n, seed=seed, edge=(24, 44), particles=(1, 4), centers=(2, 4),
                     walkers=(2000, 6000), steps=32)


def _state(sim, with_f=True):
    pos, x0 = sim.walkers_by_id()
    return dict(f=sim.populations() if with_f else None, u=sim.velocity(), c=sim.concentration(), pos=pos, x0=x0,
                m=sim.walker_moments(), mm=sim.mass_momentum(), t=sim.t)


def _same(a, b, label, regrouped=False):
    """Per-cell and per-walker results bit for bit; FP64 sums to 1e-12 relative. With
    `regrouped` (another LBM block size) the mass/momentum sums add binary32 partial sums of
    other blocks of cells: each partial over <= 256 cells carries <= 256 * 2^-24 of its
    absolute sum, and the absolute sums are at most the mass (|rho u| < rho), so the bound is
    2 * 256 * 2^-24 * mass for every entry."""
    for k in ("f", "u", "c", "pos", "x0"):
        assert np.array_equal(a[k], b[k]), f"{label}: {k} differs"
    assert a["t"] == b["t"]
    np.testing.assert_allclose(a["m"], b["m"], rtol=1e-12, atol=1e-12 * np.max(np.abs(a["m"])), err_msg=label)
    tol = 2 * 256 * 2.0 ** -24 * abs(a["mm"][0]) if regrouped else 1e-12 * np.max(np.abs(a["mm"]))
    np.testing.assert_allclose(a["mm"], b["mm"], rtol=0, atol=tol, err_msg=label)


@pytest.mark.parametrize("mode", ["branches", "fused"])
def test_batch_equals_separate_runs(mode):
    _need_gpu()
    from paper_2308_05007_gb300.rwmi import BATCH_BRANCHES, BATCH_FUSED, Batch, RwmiError, Simulation
    ws = _small_domains()
    alone = []
    for w in ws:
        with Simulation.from_workload(w) as s:
            s.step(w.steps)
            alone.append(_state(s))
    sims = [Simulation.from_workload(w) for w in ws]
    try:
        with Batch(sims, mode=BATCH_FUSED if mode == "fused" else BATCH_BRANCHES) as b:
            with pytest.raises(RwmiError):
                b.step(ws[0].sort_interval + 1)         # not a multiple of the chunk
            b.step(ws[0].steps // 2)                    # first chunk: captured
            b.step(ws[0].steps - ws[0].steps // 2)      # then replayed
            assert b.sync() >= 0
            for k, (w, s) in enumerate(zip(ws, sims)):
                _same(alone[k], _state(s), w.name)
            # work on a context's own stream after the batch sees the batch's results
            sims[0].step(2)
            assert sims[0].t == ws[0].steps + 2
    finally:
        for s in sims:
            s.close()


def test_fused_work_split_and_autotune_change_no_result():
    """Other tiles of the fused launches (LBM block, walker chunks per block, resolve and raster
    split) and the autotuner's choice: the same per-cell and per-walker results as each domain
    stepped alone (the LBM block size regroups the binary32 partial sums of mass and momentum)."""
    _need_gpu()
    from paper_2308_05007_gb300.rwmi import BATCH_FUSED, Batch, Simulation
    ws = _small_domains(4, seed=8)
    sims = [Simulation.from_workload(w) for w in ws]
    try:
        with Batch(sims, mode=BATCH_FUSED) as b:
            b.set_tiles(lbm_block=128, walker_chunks_per_block=4, resolve_walkers_per_block=2048,
                        raster_bricks_per_block=16)
            b.step(16)
            b.set_tiles(lbm_block=64, walker_chunks_per_block=2, resolve_walkers_per_block=32768,
                        raster_bricks_per_block=256)
            b.step(16)
            chosen = b.autotune(16)
            assert chosen["lbm_block"] in (64, 128, 256) and chosen == b.tiles
            b.step(16)
            assert b.sync() >= 0
            assert b.launch_count > 0
            for w, s in zip(ws, sims):
                t = s.t
                assert t % 16 == 0 and t > 48
                with Simulation.from_workload(w) as a:
                    a.step(t)
                    _same(_state(a), _state(s), w.name, regrouped=True)
    finally:
        for s in sims:
            s.close()


def test_fused_batch_refuses_contexts_it_cannot_run():
    """The paper's IBB coupling is not fused: asking for the fused form fails without side
    effects, and the automatic form falls back to per-context branches."""
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import BATCH_AUTO, BATCH_FUSED, Batch, RwmiError, Simulation
    ws = _small_domains(2, seed=9)
    ws[1] = I.with_(ws[1], coupling=1)
    sims = [Simulation.from_workload(w) for w in ws]
    try:
        with Batch(sims) as b:
            with pytest.raises(RwmiError, match="fused"):
                b.set_mode(BATCH_FUSED)
            b.set_mode(BATCH_AUTO)
            b.step(16)
            assert b.sync() >= 0
    finally:
        for s in sims:
            s.close()


def _trajectory_against_the_oracle(sim_state, w, label):
    """The single-context trajectory tolerances (shifted binary32 storage)."""
    from oracle.oracle import Oracle
    ora = Oracle.from_workload(w)
    ora.step(w.steps)
    u_o = ora.velocity()
    rel_u = np.linalg.norm(sim_state["u"].astype(np.float64) - u_o) / np.linalg.norm(u_o)
    assert rel_u <= 1e-5, (label, rel_u)
    xo, _ = ora.walkers()
    pos = sim_state["pos"]
    cells = ora.bin_positions(pos)
    diff = (cells != ora.bin_positions(xo.astype(np.float32))).sum()
    assert diff <= max(2, 1e-3 * len(pos)), (label, diff)
    assert int(sim_state["c"].sum()) == len(pos)
    return rel_u


def test_batched_domain_against_the_oracle():
    """One domain of a fused batch, after two chunks, against the FP64 oracle."""
    _need_gpu()
    from paper_2308_05007_gb300.rwmi import BATCH_FUSED, Batch, Simulation
    ws = _small_domains(3, seed=10)
    sims = [Simulation.from_workload(w) for w in ws]
    try:
        with Batch(sims, mode=BATCH_FUSED) as b:
            b.step(ws[0].steps)
            assert b.sync() >= 0
        k = int(np.argmin([w.n_cells for w in ws]))
        print("batched domain vs oracle: rel_u", _trajectory_against_the_oracle(_state(sims[k]), ws[k], ws[k].name))
    finally:
        for s in sims:
            s.close()


def test_batch_rejects_contexts_off_the_chunk_boundary():
    _need_gpu()
    from paper_2308_05007_gb300.rwmi import Batch, RwmiError, Simulation
    ws = _small_domains(2, seed=6)
    sims = [Simulation.from_workload(w) for w in ws]
    try:
        sims[1].step(1)
        with Batch(sims) as b:
            with pytest.raises(RwmiError, match="chunk boundary"):
                b.step(16)
    finally:
        for s in sims:
            s.close()


def test_autotuned_block_size_changes_no_result():
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.ragged(n_walkers=3000)
    ref = None
    for blk in (64, 128, 256):
        with Simulation.from_workload(w, lbm_block=blk) as s:
            s.step(12)
            st = _state(s)
        if ref is None:
            ref = st
        else:
            _same(ref, st, f"block {blk}", regrouped=True)
    with Simulation.from_workload(w) as s:
        picked = s.autotune()
        assert picked in (64, 128, 256)
        s.step(12)
        _same(ref, _state(s), "autotuned", regrouped=True)


def test_overlapped_raster_changes_no_result():
    """The overlapped schedules (raster of t+1 beside the LBM of t; walkers of t beside the
    fluid of t+1) give the serial schedule's results bit for bit, eager and graph-replayed."""
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation
    w = I.with_(I.ragged(n_walkers=4000), sort_interval=4, moment_interval=2)
    out = {}
    for overlap in (0, 1, 2):
        for graphs in (False, True):
            with Simulation.from_workload(w, overlap=overlap, use_graphs=graphs) as s:
                s.step(13)
                st = _state(s)
                st["solid"] = s.solid()
                st["forces"] = s.particle_forces()
                st["series"] = s.moment_series()
            out[(overlap, graphs)] = st
    ref = out[(0, False)]
    for key, st in out.items():
        _same(ref, st, f"overlap={key[0]} graphs={key[1]}")
        for a, b in zip(ref["solid"], st["solid"]):
            assert np.array_equal(a, b)
        np.testing.assert_allclose(ref["forces"], st["forces"], rtol=1e-12,
                                   atol=1e-12 * np.max(np.abs(ref["forces"])))
        assert ref["series"].shape == st["series"].shape == (6, 14)
        assert np.array_equal(ref["series"][:, 0], np.arange(2, 14, 2))   # the row of each step
        np.testing.assert_allclose(ref["series"], st["series"], rtol=1e-12, atol=1e-12)


def test_query_and_footprint():
    torch = _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation, footprint
    w = I.with_(I.oscillator(n=128, n_particles=8, n_walkers=1_000_000), sort_interval=16)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = Simulation.from_workload(w)
    s.step(64)
    free1 = torch.cuda.mem_get_info()[0]
    used = free0 - free1
    fp = footprint(w.dims, w.q, w.storage, w.n_walkers, w.metaballs.n_particles, w.metaballs.n_centers)
    # the estimate covers what the context holds, give or take the allocator's granularity
    assert used <= fp + (64 << 20), (used, fp)
    assert fp <= 1.25 * used + (64 << 20), (used, fp)
    s.step(256)
    seen_busy = s.busy()
    s.sync()
    assert not s.busy()
    assert isinstance(seen_busy, bool)
    s.close()


def test_served_results_equal_alone_and_in_the_mix():
    _need_gpu()
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation
    from paper_2308_05007_gb300.serve import Server, gpu_backend

    reqs = I.served(n_requests=6, rate=200.0, seed=11, edge=(24, 56), walkers=(1000, 20000),
                    steps=(32, 160), storage=(1, 2))

    def collect(sim, w):
        return _state(sim, with_f=False)

    srv = Server(gpu_backend(collect), budget_bytes=1 << 34, max_active=4, chunk_cell_updates=24 ** 3 * 16)
    rep = srv.run(reqs)
    assert rep.peak_active >= 2, "the requests never overlapped"
    assert len(rep.done()) == len(reqs)
    for r, rec in zip(sorted(reqs, key=lambda r: r.arrival), rep.records):
        assert rec.rid == r.rid
        with Simulation.from_workload(r.workload) as s:
            s.step(r.workload.steps)
            alone = collect(s, r.workload)
        mixed = rec.result
        for k in ("u", "c", "pos", "x0"):
            assert np.array_equal(alone[k], mixed[k]), f"request {r.rid}: {k} differs"
        assert alone["t"] == mixed["t"] == r.workload.steps
        np.testing.assert_allclose(alone["m"], mixed["m"], rtol=1e-12, atol=1e-12 * np.max(np.abs(alone["m"])))
    s = rep.summary()
    assert s["requests"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    # one served request (the smallest binary32-shifted one) against the FP64 oracle
    pick = min((r for r in reqs if r.workload.storage == 1), key=lambda r: r.workload.n_cells)
    rec = next(x for x in rep.records if x.rid == pick.rid)
    print("served request vs oracle: rel_u", _trajectory_against_the_oracle(rec.result, pick.workload, f"request {pick.rid}"))
