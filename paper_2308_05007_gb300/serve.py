"""Continuous-batching request loop over simulation contexts.

Requests (a Workload each, with an arrival time) come in as a stream. Each one that is admitted
gets its own context (librwmi.so) on its own CUDA stream. Its populations, walkers and particle
tables stay resident in HBM until it finishes. The loop admits waiting requests in arrival order
while a slot is free and the device-memory budget holds their footprint (rwmi_footprint). It
keeps every admitted context fed with chunks of steps, polls completion without blocking
(rwmi_query), and collects, closes and frees each finished request so the next ones get in. Work
of the admitted contexts overlaps on the device. Every context's result is the same as when it
runs alone, because contexts share no device state.

A request whose context fails (its creation, a step, a poll or the collection raises, e.g. an
RWMI_E_OOM the footprint did not foresee) is closed and recorded with its error; its memory
returns to the budget and the other requests carry on untouched.

The scheduler itself is plain host logic. The backend (how to make a context, its footprint, its
chunk length, what to collect) is a parameter, so the same loop runs against a fake backend in
CPU tests.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass
from typing import Callable, Optional

import numpy as np


@dataclass
class Backend:
    """How the loop talks to contexts.

    make(workload) -> sim. The sim has step(n) (asynchronous), busy() -> bool (non-blocking)
    and close(). footprint(workload) -> device bytes. chunk(workload) -> steps that one
    rwmi_step call must be a multiple of. collect(sim, workload) -> result dict, called once the
    sim is idle after its last step.
    """
    make: Callable
    footprint: Callable
    chunk: Callable
    collect: Callable


def gpu_backend(collect: Optional[Callable] = None) -> Backend:
    """The librwmi.so backend: each request is a Simulation with the context's own stream."""
    from . import rwmi

    def make(w):
        return rwmi.Simulation.from_workload(w)

    def footprint(w):
        mb = w.metaballs
        P = mb.n_particles if mb is not None else 0
        Nc = mb.n_centers if mb is not None else 0
        return rwmi.footprint(w.dims, w.q, w.storage, w.n_walkers, P, Nc)

    def chunk(w):
        L = 2
        for k in (w.sort_interval, w.moment_interval):
            if k > 0:
                L = L * k // math.gcd(L, k)
        return L

    return Backend(make, footprint, chunk, collect or default_collect)


def default_collect(sim, w) -> dict:
    """Final concentration (walkers per cell), walker moments and the FP64 mass/momentum sums."""
    return dict(concentration=sim.concentration(), moments=sim.walker_moments(),
                mass_momentum=sim.mass_momentum(), t=sim.t)


@dataclass
class Record:
    rid: int
    arrival: float              # seconds after the loop started
    cells: int
    walkers: int
    steps: int
    storage: int
    footprint: int
    admitted: float = math.nan
    finished: float = math.nan
    cancelled: bool = False
    result: Optional[dict] = None
    error: Optional[str] = None     # set when the request's context failed

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def wait(self) -> float:
        return self.admitted - self.arrival


@dataclass
class _Slot:
    rec: Record
    w: object
    sim: object
    left: int
    chunk: int


@dataclass
class Report:
    records: list
    makespan: float
    peak_bytes: int
    peak_active: int

    def done(self):
        return [r for r in self.records if not r.cancelled and not math.isnan(r.finished)]

    def summary(self) -> dict:
        d = self.done()
        lat = np.array([r.latency for r in d]) if d else np.zeros(1)
        wait = np.array([r.wait for r in d]) if d else np.zeros(1)
        cu = sum(r.cells * r.steps for r in d)
        ws = sum(r.walkers * r.steps for r in d)
        span = max(self.makespan, 1e-12)
        out = dict(requests=len(d), cancelled=sum(r.cancelled for r in self.records),
                   failed=sum(r.error is not None for r in self.records),
                   p50_latency_s=float(np.percentile(lat, 50)), p99_latency_s=float(np.percentile(lat, 99)),
                   p50_wait_s=float(np.percentile(wait, 50)), p99_wait_s=float(np.percentile(wait, 99)),
                   makespan_s=self.makespan, mlups=cu / span / 1e6, walker_steps_per_s=ws / span,
                   peak_bytes=self.peak_bytes, peak_active=self.peak_active)
        for st in sorted({r.storage for r in d}):
            sub = [r for r in d if r.storage == st]
            out[f"storage{st}_requests"] = len(sub)
            out[f"storage{st}_cell_updates"] = int(sum(r.cells * r.steps for r in sub))
        return out


class Server:
    """The request loop.

    budget_bytes: device memory the admitted contexts may hold together (sum of footprints).
    max_active: slots, i.e. contexts resident at once.
    chunk_cell_updates: cells x steps per rwmi_step call of one context (rounded to its chunk);
    it sets how often the loop revisits a context, not the results.
    """

    def __init__(self, backend: Optional[Backend] = None, budget_bytes: int = 64 << 30,
                 max_active: int = 16, chunk_cell_updates: float = 5e8, poll_s: float = 2e-4,
                 clock: Callable = time.perf_counter, sleep: Callable = time.sleep):
        self.backend = backend or gpu_backend()
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.chunk_cell_updates = float(chunk_cell_updates)
        self.poll_s = float(poll_s)
        self.clock = clock
        self.sleep = sleep
        self._cancel = set()

    def cancel(self, rid: int):
        """Drops a request: before admission it is never started; once admitted its context is
        closed at the next poll (between chunks; nothing in flight is interrupted)."""
        self._cancel.add(int(rid))

    def _chunk_steps(self, rec: Record, L: int) -> int:
        k = max(1, int(self.chunk_cell_updates // max(rec.cells, 1)))
        return max(L, k // L * L)

    def run(self, requests, time_scale: float = 1.0, on_event: Optional[Callable] = None) -> Report:
        """Serves `requests` (objects with rid, arrival in seconds, workload) and returns when
        every one has finished or was cancelled. Arrivals are replayed on the loop's clock,
        scaled by time_scale. on_event(kind, record) is called on admit, finish, cancel, reject
        and fail."""
        be = self.backend
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue: deque = deque()
        active: list = []
        records = []
        used = peak = peak_active = 0
        t0 = self.clock()

        def now():
            return self.clock() - t0

        def emit(kind, rec):
            if on_event is not None:
                on_event(kind, rec)

        def failed(rec, sim, exc):
            """Closes a failed context (best effort) and records why; the caller frees its budget."""
            rec.error = f"{type(exc).__name__}: {exc}"
            if sim is not None:
                try:
                    sim.close()
                except Exception:
                    pass
            emit("fail", rec)

        while pending or queue or active:
            progressed = False
            t = now()
            while pending and pending[0].arrival * time_scale <= t:
                r = pending.popleft()
                w = r.workload
                rec = Record(r.rid, r.arrival * time_scale, w.n_cells, int(w.n_walkers), int(w.steps),
                             int(w.storage), int(be.footprint(w)))
                records.append(rec)
                queue.append((rec, w))
                progressed = True
            # cancellations before admission
            if self._cancel and queue:
                keep = deque()
                for rec, w in queue:
                    if rec.rid in self._cancel:
                        rec.cancelled = True
                        emit("cancel", rec)
                    else:
                        keep.append((rec, w))
                queue = keep
            # admission in arrival order, while a slot and the memory budget allow
            while queue and len(active) < self.max_active:
                rec, w = queue[0]
                if rec.footprint > self.budget:          # can never fit: reject
                    queue.popleft()
                    rec.cancelled = True
                    emit("reject", rec)
                    continue
                if used + rec.footprint > self.budget:
                    break
                queue.popleft()
                try:
                    sim = be.make(w)
                except Exception as exc:
                    failed(rec, None, exc)
                    progressed = True
                    continue
                rec.admitted = now()
                used += rec.footprint
                peak = max(peak, used)
                active.append(_Slot(rec, w, sim, rec.steps, 0))
                active[-1].chunk = self._chunk_steps(rec, be.chunk(w))
                peak_active = max(peak_active, len(active))
                emit("admit", rec)
                progressed = True
            # feed idle contexts, retire finished ones
            still = []
            for s in active:
                if s.rec.rid in self._cancel:
                    s.sim.close()
                    s.rec.cancelled = True
                    used -= s.rec.footprint
                    emit("cancel", s.rec)
                    progressed = True
                    continue
                try:
                    if s.sim.busy():
                        still.append(s)
                        continue
                    if s.left > 0:
                        n = min(s.chunk, s.left)
                        s.sim.step(n)
                        s.left -= n
                        still.append(s)
                        progressed = True
                        continue
                    result = be.collect(s.sim, s.w)
                except Exception as exc:
                    failed(s.rec, s.sim, exc)
                    used -= s.rec.footprint
                    progressed = True
                    continue
                s.rec.result = result
                s.sim.close()
                s.rec.finished = now()
                used -= s.rec.footprint
                emit("finish", s.rec)
                progressed = True
            active = still
            if not progressed:
                self.sleep(self.poll_s)
        done = [r for r in records if not math.isnan(r.finished)]
        span = (max(r.finished for r in done) - min(r.arrival for r in done)) if done else 0.0
        return Report(records, span, peak, peak_active)
