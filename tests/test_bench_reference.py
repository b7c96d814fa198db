"""The reference arm of bench.py (the FP64 oracle timed on the host cores) keeps the JSON
contract: W warm-up and K timed steps as asked, each a bounded sample of the workload, one line
printed by rank 0 with the arm's own metric, unit and config."""
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line_follows_the_contract():
    a = bench.parse(["--impl", "reference", "--n", "64", "--particles", "1", "--walkers", "20000",
                     "--steps", "5", "--warmup", "3", "--reference-budget", "2"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(a, 0)
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "MLUPS"
    assert d["steps"] == 5 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert abs(d["value"] - 64 ** 3 / (d["ms_per_step"] * 1e3)) < 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "3 + 5 steps" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"] == bench.config_dict(a, bench.workload(a))
