"""bench.py's reference arm (the oracle timed on the host cores) prints the
contract's JSON line; run on CPU on a small workload with a short budget."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,sizes", [
    ("gather", ["--ref-bp", "2000000", "--reads", "4000"]),
    ("mixed", ["--scan-ref-bp", "4000000", "--mixed-reads", "3000"]),
    ("fullscan", ["--scan-ref-bp", "6000000", "--scan-reads", "512"])])
def test_reference_arm_json_line(workload, sizes):
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3", "--workload", workload,
           "--ref-seconds", "3", *sizes]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]
    # the same workload-defining keys as the GPU arm's config
    assert d["config"]["parallelism"].startswith("replicas")
    assert set(d["config"]) == {"ref_bp", "q", "bin_len", "overlap", "n_bins", "reads_per_gpu", "read_len", "E", "sub",
                                "indel", "repeat_frac", "l2", "parallelism", "workload"}
