"""Request loop host logic (no GPU): admission by footprint and slots, FIFO order, chunking,
cancellation, latency bookkeeping. The backend is a fake whose contexts take a set time per
cell-update on a fake clock."""
import math
from dataclasses import dataclass

import pytest

from paper_2308_05007_gb300 import inputs as I
from paper_2308_05007_gb300.serve import Backend, Server


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeSim:
    """Busy for cells*n*cost seconds after step(n); records what it was asked to do."""

    def __init__(self, w, clock, cost, log):
        self.w, self.clock, self.cost, self.log = w, clock, cost, log
        self.until = 0.0
        self.steps = 0
        self.closed = False

    def step(self, n):
        assert not self.closed
        start = max(self.clock(), self.until)
        self.until = start + self.w.n_cells * n * self.cost
        self.steps += n
        self.log.append(("step", self.w.name, n))

    def busy(self):
        return self.clock() < self.until

    def close(self):
        self.closed = True
        self.log.append(("close", self.w.name))


def fake_backend(clock, cost=1e-9, fp=lambda w: w.n_cells * 100, chunk=16):
    log, sims = [], {}

    def make(w):
        s = FakeSim(w, clock, cost, log)
        sims[w.name] = s
        log.append(("make", w.name))
        return s

    return Backend(make=make, footprint=fp, chunk=lambda w: chunk,
                   collect=lambda s, w: dict(steps=s.steps)), log, sims


@dataclass
class Req:
    rid: int
    arrival: float
    workload: object


def req(rid, arrival, n, steps):
    return Req(rid, arrival, I.Workload(name=f"r{rid}", dims=(n, n, n), tau=0.8, D=0.01, seed=rid,
                                        steps=steps, n_walkers=10))


def test_every_request_runs_exactly_its_steps_in_chunks():
    clk = Clock()
    be, log, sims = fake_backend(clk)
    reqs = [req(0, 0.0, 32, 100), req(1, 0.01, 48, 64), req(2, 0.02, 40, 16)]
    srv = Server(be, budget_bytes=1 << 40, max_active=4, chunk_cell_updates=32 ** 3 * 40,
                 clock=clk, sleep=clk.sleep)
    rep = srv.run(reqs)
    assert [r.result["steps"] for r in rep.records] == [100, 64, 16]
    assert all(s.closed for s in sims.values())
    # every call but the last is a whole multiple of the chunk
    steps_r0 = [n for kind, *rest in log if kind == "step" and rest[0] == "r0" for n in rest[1:]]
    assert steps_r0[:-1] and all(n % 16 == 0 for n in steps_r0[:-1]) and sum(steps_r0) == 100
    for r in rep.records:
        assert r.admitted >= r.arrival and r.finished > r.admitted
        assert math.isclose(r.latency, r.finished - r.arrival)


def test_admission_holds_the_memory_budget_and_slots():
    clk = Clock()
    be, log, sims = fake_backend(clk)
    reqs = [req(i, 0.001 * i, 48, 64) for i in range(8)]
    fp = 48 ** 3 * 100
    events = []
    srv = Server(be, budget_bytes=3 * fp, max_active=2, clock=clk, sleep=clk.sleep)
    active = set()
    peak = [0]

    def on_event(kind, rec):
        events.append((kind, rec.rid))
        if kind == "admit":
            active.add(rec.rid)
        elif kind in ("finish", "cancel"):
            active.discard(rec.rid)
        peak[0] = max(peak[0], len(active))

    rep = srv.run(reqs, on_event=on_event)
    assert peak[0] == 2 and rep.peak_active == 2
    assert rep.peak_bytes <= 3 * fp
    # FIFO: admitted in arrival order
    admits = [rid for k, rid in events if k == "admit"]
    assert admits == list(range(8))
    srv2 = Server(fake_backend(clk)[0], budget_bytes=int(1.5 * fp), max_active=8, clock=clk, sleep=clk.sleep)
    rep2 = srv2.run([req(i, 0.0, 48, 32) for i in range(4)])
    assert rep2.peak_active == 1 and len(rep2.done()) == 4


def test_too_large_request_is_rejected_not_deadlocked():
    clk = Clock()
    be, log, sims = fake_backend(clk)
    srv = Server(be, budget_bytes=40 ** 3 * 100, max_active=4, clock=clk, sleep=clk.sleep)
    rep = srv.run([req(0, 0.0, 64, 16), req(1, 0.0, 32, 16)])
    assert rep.records[0].cancelled and math.isnan(rep.records[0].finished)
    assert rep.records[1].result["steps"] == 16


def test_cancel_before_and_after_admission():
    clk = Clock()
    be, log, sims = fake_backend(clk, cost=1e-8)
    srv = Server(be, budget_bytes=1 << 40, max_active=1, chunk_cell_updates=32 ** 3 * 16,
                 clock=clk, sleep=clk.sleep)

    def on_event(kind, rec):
        if kind == "admit" and rec.rid == 0:
            srv.cancel(0)     # cancelled while running
            srv.cancel(2)     # cancelled while waiting

    rep = srv.run([req(0, 0.0, 32, 1600), req(1, 0.0, 32, 32), req(2, 0.0, 32, 32)], on_event=on_event)
    r0, r1, r2 = rep.records
    assert r0.cancelled and sims["r0"].closed and sims["r0"].steps < 1600
    assert r2.cancelled and "r2" not in sims
    assert not r1.cancelled and r1.result["steps"] == 32
    s = rep.summary()
    assert s["requests"] == 1 and s["cancelled"] == 2


def test_poisson_stream_summary_counts_work():
    clk = Clock()
    be, log, sims = fake_backend(clk, cost=1e-10)
    reqs = I.served(n_requests=12, rate=20.0, seed=4, edge=(32, 64), walkers=(1000, 10000),
                    steps=(32, 256))
    srv = Server(be, budget_bytes=1 << 40, max_active=4, clock=clk, sleep=clk.sleep)
    rep = srv.run(reqs)
    s = rep.summary()
    assert s["requests"] == 12
    cu = sum(r.workload.n_cells * r.workload.steps for r in reqs)
    assert s["mlups"] == pytest.approx(cu / rep.makespan / 1e6)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
    # arrivals were replayed on the clock: nobody was admitted before arriving
    for r in rep.records:
        assert r.admitted >= r.arrival
    assert all(w.workload.steps % 16 == 0 for w in reqs)


def test_a_failing_request_is_closed_and_the_others_carry_on():
    """One context cannot be made (an allocation failure the footprint did not foresee), another
    fails in its second chunk and a third when its results are collected. Each is closed and
    recorded with its error, its memory returns to the budget, and every other request runs
    exactly its steps."""
    clk = Clock()
    be, log, sims = fake_backend(clk)
    make0, collect0 = be.make, be.collect

    def make(w):
        if w.name == "r1":
            raise RuntimeError("RWMI_E_OOM: dalloc: out of memory")
        s = make0(w)
        if w.name == "r2":
            step0 = s.step

            def step(n):
                if s.steps > 0:
                    raise RuntimeError("RWMI_E_CUDA: launch failed")
                step0(n)
            s.step = step
        return s

    def collect(s, w):
        if w.name == "r4":
            raise RuntimeError("RWMI_E_NONFINITE: non-finite walker velocity")
        return collect0(s, w)

    be.make, be.collect = make, collect
    fp = 32 ** 3 * 100
    events = []
    srv = Server(be, budget_bytes=2 * fp, max_active=2, chunk_cell_updates=32 ** 3 * 16,
                 clock=clk, sleep=clk.sleep)
    rep = srv.run([req(i, 0.001 * i, 32, 64) for i in range(6)],
                  on_event=lambda kind, rec: events.append((kind, rec.rid)))
    by = {r.rid: r for r in rep.records}
    assert "OOM" in by[1].error and "r1" not in sims
    assert "CUDA" in by[2].error and sims["r2"].closed and sims["r2"].steps == 16
    assert "NONFINITE" in by[4].error and sims["r4"].closed
    for rid in (0, 3, 5):
        assert by[rid].error is None and by[rid].result["steps"] == 64 and sims[f"r{rid}"].closed
    for rid in (1, 2, 4):
        assert by[rid].result is None and math.isnan(by[rid].finished) and not by[rid].cancelled
    assert sorted(rid for k, rid in events if k == "fail") == [1, 2, 4]
    assert rep.peak_bytes <= 2 * fp
    s = rep.summary()
    assert s["requests"] == 3 and s["failed"] == 3 and s["cancelled"] == 0
