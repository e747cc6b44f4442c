"""bench.py's contract on the CPU: the reference arm's JSON line (the oracle timed on the
host cores) carries every key of the measurement contract, and the algorithmic flop counts
the roofline credits are the per-node counts of the method (Eq. fde1 solved by Picard
iteration: LI 44 and EA 30 flops per node and iteration; the Matern noise 4 + 6k + 4(k - 1)
per node and step)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_flop_counts():
    n, K = 1024, 8
    assert bench.step_flops(n, K, "ea", 7, 2) == n * (30 * 7 + (2 * K + 5) * 2)
    assert bench.step_flops(n, K, "li", 7, 2) == n * (44 * 7 + 2 * K * 2)
    assert bench.matern_flops_per_node(3) == 30 and bench.matern_flops_per_node(1) == 10
    assert bench.step_flops(n, K, "ea", 7, 2, bench.matern_flops_per_node(3)) == n * (30 * 7 + (30 + 5) * 2)
    # a warm-started step's u = H^-1 M m: the mass right-hand side and one Helmholtz solve
    assert bench.FLOPS_PER_NODE_WARM_START == 3 + 9
    # adjoint window: forward (LI) + 32 per adjoint iteration + (16 + 2K) per step, N Ns steps
    assert bench._adjoint_flops(n, K, 4, 5, 100, 90) == n * (44 * 100 + 2 * K * 20) + n * (32 * 90 + (16 + 2 * K) * 20)


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.METRIC
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["higher_is_better"] is True and d["data"] == "synthetic" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
