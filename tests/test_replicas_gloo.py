"""Replica (weak-scaling) host logic of bench.py on two CPU ranks over gloo.

The path does not shard: `bench.py --gpus N` runs N independent replicas, one per rank, with no
collective on the data path. The host logic still has multi-rank parts: every rank must build
the same seeded workload, the job time is the maximum over ranks, the job value counts all
ranks' work, and the reference arm runs on rank 0 alone (the other ranks exit without work).
"""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import hashlib

    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a = bench.parse([])
        a.n, a.particles, a.walkers = 128, 4, 1000
        w = bench.workload(a)
        h = hashlib.sha256()
        for arr in (w.metaballs.origin, w.metaballs.centers_body, w.metaballs.k):
            h.update(np.ascontiguousarray(arr).tobytes())
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        rate = bench.job_rate(world, w.n_cells, 10, t)
        buf = io.StringIO()
        if rank != 0:       # rank 0 would time the oracle here: seconds of CPU work, not needed
            with contextlib.redirect_stdout(buf):
                bench.run_reference(a, rank)
        out[rank] = dict(hash=h.hexdigest(), t=t, rate=rate, ref_out=buf.getvalue())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_workload_time_and_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    assert res[0]["hash"] == res[1]["hash"], "ranks built different workloads"
    assert res[0]["t"] == res[1]["t"] == 2.5, "job time is not the max over ranks"
    assert res[0]["rate"] == pytest.approx(2 * 128 ** 3 * 10 / 2.5)
    assert res[1]["ref_out"] == "", "the reference arm printed on a rank other than 0"


def test_gpus_n_without_torchrun_relaunches_n_ranks():
    """`bench.py --gpus 2` started as one plain process re-launches itself as two ranks under
    torch.distributed.run (here the reference arm, which needs no GPU: rank 0 prints the one
    JSON line with n_gpus 2, the other rank exits without work); it never reports one GPU for
    a two-GPU request."""
    import json
    import subprocess
    sys.path.insert(0, ROOT)
    import bench

    assert bench.launch_plan(1, {}, []) is None
    assert bench.launch_plan(2, {"RANK": "0", "WORLD_SIZE": "2"}, []) is None
    with pytest.raises(SystemExit):
        bench.launch_plan(2, {"RANK": "0", "WORLD_SIZE": "1"}, [])
    plan = bench.launch_plan(2, {}, ["--gpus", "2"])
    assert plan[1:3] == ["-m", "torch.distributed.run"] and "--nproc-per-node=2" in plan
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--n", "64", "--particles", "1", "--walkers", "20000", "--steps", "2", "--warmup", "1",
                        "--reference-budget", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
