#!/usr/bin/env python3
"""Benchmark of the fused fluid-solute step (LBM stream-collide on partially-saturated cells +
random-walk advance of solute walkers) on the 256^3 oscillator workload, one GB300 per rank.

One "step" is one pass of the whole path: particle poses and brick lists, metaball
rasterisation, the fused LBM kernel, the walker advance, and -- every 16 steps -- the counting
sort/binning of walkers (concentration) and the FP64 walker moments. Inputs are resident in HBM
and larger than L2 (each population buffer is 1 GB), so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank advances its own replica
(weak scaling, no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LBM MLUPS + walker-steps/s and %HBM roofline, FP32/FP16-shift vs plain; p99 latency"
STORE_NAMES = {0: "fp32", 1: "fp32_shift", 2: "fp16_shift", 3: "fp64_shift"}
STORE_BYTES = {0: 4, 1: 4, 2: 2, 3: 8}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "lbm_kernel_oscillator_256.md")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=32)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--reference-budget", type=float, default=90.0,
                    help="seconds of oracle time for all --impl reference steps together")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--walkers", type=int, default=10_000_000)
    ap.add_argument("--particles", type=int, default=64)
    ap.add_argument("--q", type=int, default=15)
    ap.add_argument("--storage", type=int, default=1)
    ap.add_argument("--sort-interval", type=int, default=16)
    ap.add_argument("--moment-interval", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--overlap", type=int, default=2, choices=[0, 1, 2])
    ap.add_argument("--lbm-staging", type=int, default=0, choices=[0, 1],
                    help="LBM update with TMA-staged rows (1) or direct loads (0)")
    ap.add_argument("--coupling", type=int, default=0, choices=[0, 1])
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--batch-domains", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=160)
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--served-requests", type=int, default=32)
    ap.add_argument("--served-step-scale", type=float, default=0.05)
    return ap.parse_args(argv)


def workload(a):
    from paper_2308_05007_gb300 import inputs as I
    w = I.oscillator(n=a.n, n_particles=a.particles, n_walkers=a.walkers, q=a.q, storage=a.storage)
    w = I.with_(w, coupling=getattr(a, "coupling", 0))
    return I.with_(w, sort_interval=a.sort_interval, moment_interval=a.moment_interval)


def bytes_per_step(w, n_cells, s):
    """Algorithmic HBM bytes of one step: populations read + written once (2 Q s per cell), the
    velocity written by the LBM kernel and gathered once by the cell-sorted walkers (12 + 12 B
    per cell), each walker's float4 read and written (32 B). The kernels move 4 B per cell more
    each way (rho rides along in a float4, one 16-byte gather per corner); that is not counted."""
    return n_cells * (2 * w.q * s + 24) + 32 * w.n_walkers


def lbm_bytes_per_launch(w, n_cells, s):
    """Algorithmic bytes of one launch of the LBM update: 2 Q s per cell + 12 B of velocity."""
    return n_cells * (2 * w.q * s + 12)


def config_dict(a, w):
    return {
        "workload": (f"oscillator {a.n}^3 D3Q{w.q} {STORE_NAMES[w.storage]}, no-slip z-walls, tau 0.7, "
                     f"F=5e-6 sin(2 pi t/2000) x; {a.particles} metaball particles (4-8 centres, "
                     f"sigma 4, k U[20,60]) oscillating 5 sin(2 pi t/2000) x; "
                     f"{a.walkers:.0e} walkers, D=0.005"),
        "cells": w.n_cells, "walkers": w.n_walkers, "particles": a.particles, "q": w.q,
        "storage": STORE_NAMES[w.storage], "sort_interval": w.sort_interval,
        "moment_interval": w.moment_interval,
        "l2": "inputs larger than L2 (populations 2 x %.2f GB), no flush" % (w.n_cells * w.q * STORE_BYTES[w.storage] / 1e9),
        "graphs": "captured runs of up to 64 steps (whole %d-step chunks), replayed" % max(w.sort_interval, w.moment_interval, 2),
        "lbm_update": ("rows staged in shared memory by TMA tensor copies" if getattr(a, "lbm_staging", 0)
                       and w.storage in (0, 1, 2) and a.n % (8 if w.storage == 2 else 4) == 0
                       else "direct coalesced loads"),
        "schedule": {0: "serial", 1: "raster of t+1 on a second stream beside the LBM of t",
                     2: "raster of t+1 beside the LBM of t; walkers of t on a third stream beside "
                        "the fluid of t+1"}[getattr(a, "overlap", 2)],
    }


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        load = [x for x in sm if x > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                          if r[3].replace(".", "").isdigit())}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {"hbm_gbs": 6800.0, "fallback": True}


def lbm_source_digest() -> str:
    """First 16 hex digits of the SHA-256 of the LBM kernel's code (kernel + lattice header),
    with comments, trailing blanks and blank lines removed: a comment edit keeps the digest."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("rwmi_lbm.cu", "rwmi_lattice.cuh"):
        src = open(os.path.join(ROOT, "paper_2308_05007_gb300", "csrc", name)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def profiled_traffic(a):
    """Per-launch DRAM bytes of the LBM kernel from the committed ncu summary, if that summary
    was taken on this workload and on the current kernel source (else None)."""
    import hashlib
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    digest = lbm_source_digest()
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != digest or vals.get("workload_n") != str(a.n):
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(a, w):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of the same workload:
    one fluid step (solid fraction + LBM) of the full box, plus one walker step of a 1e4-walker
    sample; the full-step time is extrapolated to all walkers."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2308_05007_gb300 import inputs as I
    ws = I.with_(w, n_walkers=10000)
    t0 = time.perf_counter()
    o = Oracle.from_workload(ws)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.step_fluid(1)
    t_fluid = time.perf_counter() - t0
    x, _ = o.walkers()
    o.set_time(o.t - 1)
    t0 = time.perf_counter()
    o.walkers_advance(x, np.arange(len(x), dtype=np.uint32))
    t_walk = (time.perf_counter() - t0) * (w.n_walkers / len(x))
    t_step = t_fluid + t_walk
    return {
        "value": w.n_cells / t_step / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
        "walker_steps_per_s": w.n_walkers / t_step,
        "sample": (f"1 fluid step of the full {a.n}^3 box ({t_fluid:.1f} s) + 1 walker step of 1e4 "
                   f"walkers ({t_walk * len(x) / w.n_walkers:.2f} s), walker time scaled to "
                   f"{w.n_walkers:.0e}; setup {t_setup:.1f} s untimed"),
        "s_per_step": t_step,
    }


def oracle_sampled_steps(a, w, steps: int, warmup: int, budget_s: float = 90.0):
    """The FP64 oracle as it stands, single-threaded, over `warmup` + `steps` bounded samples of the
    workload, one per step. A sample is whole x-rows of cells at random (y, z): their solid
    fraction at t+1 and their LBM update at t, as one step computes them. It also holds a slice
    of walkers, about the workload's walkers per cell, advanced by one step. The sample's time is
    scaled to the full box and the full walker count. The sample size is set by a short untimed
    probe so that all steps together take about `budget_s` seconds."""
    import numpy as np
    from oracle.oracle import Oracle
    from paper_2308_05007_gb300 import inputs as I
    pool = 10000
    o = Oracle.from_workload(I.with_(w, n_walkers=pool))
    n0, n1, n2 = w.dims
    t = o.t
    o.lbm_cells(np.zeros(1, np.int64))            # solid fraction at t for the LBM sample (untimed)
    xw, _ = o.walkers()
    ids_all = np.arange(pool, dtype=np.uint32)
    per_cell = w.n_walkers / w.n_cells
    rng = np.random.default_rng(w.seed + 17)

    def sample(rows):
        jk = rng.integers(0, n1 * n2, rows)
        cells = (jk[:, None] * n0 + np.arange(n0)[None, :]).reshape(-1).astype(np.int64)
        nw = int(min(pool, max(1, round(per_cell * len(cells)))))
        w0 = int(rng.integers(0, pool - nw + 1))
        t0 = time.perf_counter()
        o.solid_cells(cells, t + 1)
        o.lbm_cells(cells)
        t1 = time.perf_counter()
        o.walkers_advance(xw[w0:w0 + nw], ids_all[w0:w0 + nw])
        t2 = time.perf_counter()
        return (t1 - t0) * (w.n_cells / len(cells)) + (t2 - t1) * (w.n_walkers / nw), len(cells), nw

    probe_rows = 8
    t_probe = time.perf_counter()
    sample(probe_rows)
    t_probe = time.perf_counter() - t_probe
    target = min(max(budget_s / max(steps + warmup, 1), 0.02), 5.0)
    rows = int(min(n1 * n2, max(1, probe_rows * target / max(t_probe, 1e-6))))
    for _ in range(warmup):
        sample(rows)
    est = []
    for _ in range(steps):
        ts, nc, nw = sample(rows)
        est.append(ts)
    t_step = float(np.mean(est))
    return {
        "value": w.n_cells / t_step / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
        "walker_steps_per_s": w.n_walkers / t_step,
        "sample": (f"{warmup} + {steps} steps, each {rows} random x-rows ({nc} cells: solid fraction "
                   f"and LBM update) + {nw} walkers; each step's time scaled to the full "
                   f"{n0}x{n1}x{n2} box and {w.n_walkers:.0e} walkers"),
        "s_per_step": t_step,
    }


def run_reference(a, rank):
    if rank != 0:
        return
    w = workload(a)
    cb = oracle_sampled_steps(a, w, a.steps, a.warmup, a.reference_budget)
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": cb["s_per_step"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(a, w),
        "walker_steps_per_s": cb["walker_steps_per_s"],
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "FP64 CPU oracle as the reference arm; ms_per_step is the full step extrapolated from the samples",
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist, device) -> float:
    """The maximum of a per-rank number over all ranks: the slowest replica sets the job time."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed units_per_rank per step."""
    return world * units_per_rank * steps / seconds


def measure_variants(a, stream):
    """The same workload with the other population storages (plain binary32, binary32 shifted by
    w_i rho0, binary16 shifted, binary64 shifted with binary64 arithmetic) and velocity sets
    (D3Q15, the paper's D3Q19): per-phase GPU time of 16 eager steps (CUDA events), LBM kernel
    HBM fraction and whole-step MLUPS. The binary64 run is bound by GB300's FP64 rate, not HBM.
    Then the paper's IBB coupling in place of partially saturated cells, and free particles (the
    DEM of Eqs. 4-11) in place of the prescribed motion (graph-replayed step time as well)."""
    import argparse as _ap

    import numpy as np
    import torch
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation
    peak = float(measured_peaks()["hbm_gbs"])
    out = {}
    for q in (15, 19):
        for storage, staging in ((0, 0), (1, 0), (2, 0), (3, 0), (0, 1), (1, 1), (2, 1)):
            b = _ap.Namespace(**vars(a))
            b.q, b.storage = q, storage
            w = workload(b)
            sim = Simulation.from_workload(w, seed_walkers=False, lbm_staging=staging)
            sim.set_stream(stream)
            sim.seed_walkers(w.n_walkers, *w.walker_box)
            sim.step(16)
            ph = sim.step_timed(16)
            one = sorted(sim.step_timed(1)["lbm"] for _ in range(5))[2]
            sim.close()
            s_bytes = STORE_BYTES[storage]
            lbm_ms = (ph["lbm"] - one) / 15   # the update alone (16 updates + 1 reduce pass)
            step_ms = sum(ph.values()) / 16
            gbs = lbm_bytes_per_launch(w, w.n_cells, s_bytes) / (lbm_ms / 1e3) / 1e9
            name = f"D3Q{q}_{STORE_NAMES[storage]}" + ("_tma" if staging else "")
            out[name] = {
                "lbm_ms": lbm_ms, "lbm_gbs": gbs, "lbm_hbm_frac": gbs / peak,
                "step_ms_eager": step_ms, "mlups_eager": w.n_cells / (step_ms / 1e3) / 1e6}
    # the paper's own coupling (IBB + momentum exchange + refilling) instead of partially
    # saturated cells, binary32 shifted storage; its LBM phase includes the node classification
    for q in (15, 19):
        b = _ap.Namespace(**vars(a))
        b.q, b.storage = q, 1
        w = I.with_(workload(b), coupling=1)
        sim = Simulation.from_workload(w, seed_walkers=False)
        sim.set_stream(stream)
        sim.seed_walkers(w.n_walkers, *w.walker_box)
        sim.step(16)
        ph = sim.step_timed(16)
        sim.step(32)
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(64)
            e1.record(stream)
            torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / 64
        sim.close()
        lbm_ms = ph["lbm"] / 16
        gbs = lbm_bytes_per_launch(w, w.n_cells, 4) / (lbm_ms / 1e3) / 1e9
        out[f"D3Q{q}_fp32_shift_ibb"] = {
            "lbm_ms": lbm_ms, "lbm_gbs": gbs, "lbm_hbm_frac": gbs / peak,
            "step_ms": step_ms, "mlups": w.n_cells / (step_ms / 1e3) / 1e6}
    # every particle's force and torque recorded on every step (force_interval 1): each step then
    # runs the fused update-and-reduce pass that the headline runs on 1 step in 16
    b = _ap.Namespace(**vars(a))
    b.q, b.storage = 15, 1
    w = workload(b)
    sim = Simulation.from_workload(w, seed_walkers=False, force_interval=1)
    sim.set_stream(stream)
    sim.seed_walkers(w.n_walkers, *w.walker_box)
    sim.step(64)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(128)
        e1.record(stream)
        torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 128
    rows, _ = sim.force_series(max_rows=128)
    sim.close()
    out["D3Q15_fp32_shift_forces_every_step"] = {
        "step_ms": step_ms, "mlups": w.n_cells / (step_ms / 1e3) / 1e6, "rows_recorded": int(len(rows))}
    # free particles (Eqs. 4-11) in place of the prescribed motion: the same box and particles,
    # density 2, gravity, damped frictional contacts, 10 DEM steps per LBM step; the LBM forms the
    # force in its update on every step, and the raster of t+1 follows the DEM
    w = I.oscillator_dem(n=a.n, n_particles=a.particles, n_walkers=a.walkers, q=15, storage=1)
    w = I.with_(w, sort_interval=a.sort_interval, moment_interval=a.moment_interval)
    sim = Simulation.from_workload(w, seed_walkers=False)
    sim.set_stream(stream)
    sim.seed_walkers(w.n_walkers, *w.walker_box)
    sim.step(16)
    ph = sim.step_timed(16)
    sim.step(32)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(64)
        e1.record(stream)
        torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 64
    st = sim.particle_state()
    sim.close()
    lbm_ms = ph["lbm"] / 16
    gbs = lbm_bytes_per_launch(w, w.n_cells, 4) / (lbm_ms / 1e3) / 1e9
    out["D3Q15_fp32_shift_dem"] = {
        "lbm_ms": lbm_ms, "lbm_gbs": gbs, "lbm_hbm_frac": gbs / peak,
        "dem_and_poses_ms": ph["pose_bricks"] / 16, "substeps": w.dem.substeps,
        "step_ms": step_ms, "mlups": w.n_cells / (step_ms / 1e3) / 1e6,
        "max_particle_speed": float(np.linalg.norm(st[:, 7:10], axis=1).max())}
    # the paper's own pairing: free particles with IBB, momentum exchange and refilling
    wi = I.with_(w, coupling=1)
    sim = Simulation.from_workload(wi, seed_walkers=False)
    sim.set_stream(stream)
    sim.seed_walkers(wi.n_walkers, *wi.walker_box)
    sim.step(16)
    ph = sim.step_timed(8)
    sim.step(8)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(32)
        e1.record(stream)
        torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 32
    sim.close()
    out["D3Q15_fp32_shift_ibb_dem"] = {
        "lbm_ms": ph["lbm"] / 8, "dem_and_poses_ms": ph["pose_bricks"] / 8, "step_ms": step_ms,
        "mlups": wi.n_cells / (step_ms / 1e3) / 1e6}
    return out


def measure_precision_case(a):
    """The precision workload at full size: 384^3 periodic box (parity physics: tau 0.8, constant
    body force 1e-6 along x), 128 static particles, 3e7 walkers, for each population storage.
    Whole-step throughput over graph-replayed steps (CUDA events on the context's stream after a
    warm-up), and the step's algorithmic bytes against the measured HBM peak."""
    import torch
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import Simulation
    peak = float(measured_peaks()["hbm_gbs"])
    out = {}
    base = I.precision(n=384, n_particles=128, n_walkers=30_000_000, seed=2)
    base = I.with_(base, sort_interval=16, moment_interval=16)
    stream = torch.cuda.Stream()
    for storage in (1, 0, 2, 3):
        w = I.with_(base, storage=storage)
        sim = Simulation.from_workload(w, seed_walkers=False)
        sim.set_stream(stream)
        sim.seed_walkers(w.n_walkers, *w.walker_box)
        n = 16 if storage == 3 else 48
        with torch.cuda.stream(stream):
            sim.step(16)
            assert sim.sync() >= 0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(n)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / n
            assert sim.sync() >= 0
        sim.close()
        sb = STORE_BYTES[storage]
        step_bytes = bytes_per_step(w, w.n_cells, sb)
        out[STORE_NAMES[storage]] = {"ms_per_step": ms, "mlups": w.n_cells / (ms / 1e3) / 1e6,
                                     "walker_steps_per_s": w.n_walkers / (ms / 1e3),
                                     "step_hbm_frac": step_bytes / (ms / 1e3) / 1e9 / peak, "steps": n}
    return {"workload": "384^3 periodic, tau 0.8, F=1e-6 x, 128 static metaball particles, 3e7 walkers, "
                        "D=0.01, D3Q15", "cells": base.n_cells, "walkers": base.n_walkers, "storages": out}


def measure_batched(a):
    """Independent periodic domains advanced together, two mixes: the batched workload (64
    domains, edges U{48..160}, 4-32 particles of 2-10 centres, 1e5-2e6 walkers, tau U[0.6, 1],
    D U[0.001, 0.02]) and 256 small domains (edges U{16..48}, 1-4 particles of 2-4 centres,
    2e3-4e4 walkers), where launch gaps dominate. Each mix three ways: "fused" (one launch per
    phase for all domains, tiles picked by rwmi_batch_autotune), "branches" (one graph of
    per-domain branches per chunk) and "separate" (each domain's own rwmi_step on its own
    stream, LBM block size from rwmi_autotune). Whole-job MLUPS by host wall clock around the
    launches and a final synchronisation, after a warm-up that captures every graph."""
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.rwmi import BATCH_BRANCHES, BATCH_FUSED, Batch, Simulation
    mixes = {
        "domains_64": dict(n_domains=a.batch_domains, seed=3),
        "small_256": dict(n_domains=256, seed=7, edge=(16, 48), particles=(1, 4), centers=(2, 4),
                          walkers=(2000, 40000)),
    }
    out = {}
    for label, kw in mixes.items():
        ws = I.batched(**kw)
        sims = [Simulation.from_workload(w) for w in ws]
        blocks = [s.autotune() for s in sims]
        cells = sum(w.n_cells for w in ws)
        walkers = sum(w.n_walkers for w in ws)
        n = max(16, a.batch_steps // 16 * 16)
        res = {"domains": len(ws), "cells": cells, "walkers": walkers, "steps": n,
               "edges": [min(w.dims[0] for w in ws), max(w.dims[0] for w in ws)],
               "lbm_block_histogram": {str(b): blocks.count(b) for b in sorted(set(blocks))}}

        def rate(dt):
            return {"mlups": cells * n / dt / 1e6, "walker_steps_per_s": walkers * n / dt, "ms_per_step": dt / n * 1e3}

        for mode in ("fused", "branches"):
            with Batch(sims, mode=BATCH_FUSED if mode == "fused" else BATCH_BRANCHES) as b:
                if mode == "fused":
                    res["fused_tiles"] = b.autotune(16)
                b.step(32)
                b.sync()
                l0 = b.launch_count
                t0 = time.perf_counter()
                b.step(n)
                assert b.sync() >= 0
                dt = time.perf_counter() - t0
                res[mode] = rate(dt)
                if mode == "fused":
                    res[mode]["launches_per_step"] = (b.launch_count - l0) / n
        for s in sims:
            s.step(32)
        for s in sims:
            s.sync()
        t0 = time.perf_counter()
        for c in range(0, n, 16):
            for s in sims:
                s.step(16)
        for s in sims:
            assert s.sync() >= 0
        res["separate"] = rate(time.perf_counter() - t0)
        for s in sims:
            s.close()
        out[label] = res
    return out


def measure_served(a):
    """Poisson request stream (20 req/s) of simulations with edges log-uniform in [32, 256],
    1e5-1e7 walkers (at most 2 per cell), FP32-shift or FP16-shift populations and
    1000-20000 steps scaled by --served-step-scale, served by the continuous-batching loop
    (admission by rwmi_footprint within half the free device memory, 16 slots)."""
    import torch
    from paper_2308_05007_gb300 import inputs as I
    from paper_2308_05007_gb300.serve import Server
    reqs = I.served(n_requests=a.served_requests, rate=20.0, seed=4, step_scale=a.served_step_scale)
    budget = int(torch.cuda.mem_get_info()[0] * 0.5)
    srv = Server(budget_bytes=budget, max_active=16)
    rep = srv.run(reqs)
    out = rep.summary()
    out.update({"rate_per_s": 20.0, "step_scale": a.served_step_scale, "budget_bytes": budget,
                "max_active": 16,
                "steps_range": [min(r.workload.steps for r in reqs), max(r.workload.steps for r in reqs)],
                "edge_range": [min(r.workload.dims[0] for r in reqs), max(r.workload.dims[0] for r in reqs)]})
    return out


def launch_plan(gpus: int, env, argv):
    """How this process runs `--gpus N`: None when it is already one of N ranks (or N = 1), else
    the command that re-launches the benchmark as N ranks under torch.distributed.run on this node
    (rendezvous on 127.0.0.1). A process started by torchrun with a different world size is an
    error, never a silent single-rank run."""
    world = int(env.get("WORLD_SIZE", "1"))
    if "RANK" in env or world > 1:
        if world != gpus:
            raise SystemExit(f"bench.py: --gpus {gpus} but WORLD_SIZE {world}")
        return None
    if gpus <= 1:
        return None
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr", "127.0.0.1", f"--master-port={port}", "--", os.path.abspath(__file__), *argv]


def main():
    a = parse()
    plan = launch_plan(a.gpus, os.environ, sys.argv[1:])
    if plan:
        sys.exit(subprocess.call(plan))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank)
        return
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2308_05007_gb300.rwmi import Simulation

    w = workload(a)
    s_bytes = STORE_BYTES[w.storage]
    stream = torch.cuda.Stream()
    sim = Simulation.from_workload(w, seed_walkers=False, overlap=a.overlap, lbm_staging=a.lbm_staging)
    sim.set_stream(stream)
    sim.seed_walkers(w.n_walkers, *w.walker_box)
    L = 16
    # Warm-up: at least W steps, then the timed step count once more from the same alignment
    # (time mod 2 L: the buffer parities and the sort phase), so that the timed region replays
    # the captured runs of steps a user's repeated calls replay; the per-phase timing runs in
    # between. Every warm-up step is a full step.
    period = 2 * L
    steps = max(a.steps, 1)
    warm = (max(a.warmup, 3) + period - 1) // period * period
    with torch.cuda.stream(stream):
        sim.step(warm)
        sim.step(steps)
        sim.step(-(warm + steps) % period)
        assert sim.sync() >= 0
        # per-phase GPU time (CUDA events on the launching stream, eager launches)
        phases = sim.step_timed(L)
        n_timed_phase_steps = L
        # the update kernel alone: a timed run of L steps holds L - 1 updates and one reducing step
        # (the fused update-and-reduce pass), a timed single step one reducing step; the reducing
        # step's extra time is reported as reduce_pass_ms
        one = sorted(sim.step_timed(1)["lbm"] for _ in range(7))[3]
        lbm_update_ms = (phases["lbm"] - one) / (L - 1)
        reduce_pass_ms = one - lbm_update_ms
        sim.step(-sim.t % period)
        warm = sim.t
        assert sim.sync() >= 0
        # the timed region
        clocks = Clocks(torch.cuda.current_device())
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        l0 = sim.launch_count
        ev0.record(stream)
        sim.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        launches = sim.launch_count - l0
        clk = clocks.stop()
        if dist:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        st = sim.sync()
        assert st >= 0, st
    ms = max_over_ranks(ms, dist, "cuda")
    sec = ms / 1e3
    mlups = job_rate(world, w.n_cells, steps, sec) / 1e6
    wsps = job_rate(world, w.n_walkers, steps, sec)

    # e2e through the public API with host buffers: H2D of the walker positions from pinned host
    # memory, the steps, D2H of the concentration field and the moments
    e2e = None
    if not a.no_e2e:
        pos, _, _ = sim.walkers(with_x0=False)
        pinned = torch.from_numpy(pos).pin_memory()
        conc = torch.empty(w.n_cells, dtype=torch.int32).pin_memory()
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            sim.set_walkers(pinned)
            sim.step(steps)
            sim.concentration(out=conc)
            mom = sim.walker_moments()
            torch.cuda.synchronize()
            te = time.perf_counter() - t0
        te = max_over_ranks(te, dist, "cuda")
        assert int(conc.sum()) == w.n_walkers and mom[0] == w.n_walkers
        e2e = {"value": job_rate(world, w.n_cells, steps, te) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": pinned.numel() * 4 / steps,
               "d2h_bytes_per_step": (conc.numel() * 4 + 13 * 8) / steps,
               "walker_steps_per_s": job_rate(world, w.n_walkers, steps, te)}

    if rank != 0:
        return
    peaks = measured_peaks()
    lbm_ms = lbm_update_ms
    achieved = lbm_bytes_per_launch(w, w.n_cells, s_bytes) / (lbm_ms / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])
    traffic = profiled_traffic(a)
    step_bytes = bytes_per_step(w, w.n_cells, s_bytes)
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": steps,
        "warmup": warm, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if w.storage == 3 else "f32", "data": "synthetic",
        "config": config_dict(a, w),
        "walker_steps_per_s": wsps,
        "step_hbm_frac": step_bytes / (ms / steps / 1e3) / 1e9 / peak,
        "step_algorithmic_bytes": step_bytes,
        "roofline": {"kernel": "lbm_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": lbm_bytes_per_launch(w, w.n_cells, s_bytes),
                     "launch_ms": lbm_update_ms, "reduce_pass_ms": reduce_pass_ms,
                     "phase_ms": phases["lbm"] / n_timed_phase_steps,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if not peaks.get("fallback") else "fallback"},
        "phase_ms_per_step": {k: v / n_timed_phase_steps for k, v in phases.items()},
        "gpu_launches": launches,
        "bricks": sim.brick_stats(),
        "counters": sim.counters(),
        "clocks": clk,
    }
    if e2e:
        line["e2e"] = e2e
    sim.close()
    if not a.no_variants:
        line["variants"] = measure_variants(a, stream)
    if not a.no_precision:
        line["precision_384"] = measure_precision_case(a)
    if not a.no_batched:
        line["batched"] = measure_batched(a)
    if not a.no_served:
        line["served"] = measure_served(a)
        line["p99_latency_s"] = line["served"]["p99_latency_s"]
    if world == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline(a, w)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
