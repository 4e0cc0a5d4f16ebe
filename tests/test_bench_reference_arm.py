"""bench.py's reference arm (the FP64 oracle timed on the host cores) on the small planar
workload, on CPU: one JSON line with the contract's keys, impl "reference", the workload's
own tolerance, and e2e / cpu_baseline describing the same run."""
import json
import os
import subprocess
import sys


def test_reference_arm_prints_one_contract_line(repo_root):
    cmd = [sys.executable, os.path.join(repo_root, "bench.py"), "--impl", "reference",
           "--workload", "planar16", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=repo_root)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    for k in ("metric", "value", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["tol"] == 1e-10 and d["config"]["ntrace"] == 6400
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
