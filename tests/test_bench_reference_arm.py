"""bench.py's reference arm (the FP64 oracle timed on the host cores) on the small planar
workload, on CPU: one JSON line with the contract's keys, impl "reference", the workload's
own tolerance and the same config dict as the GPU arm's, full solves counted honestly (at
most one warm-up), and e2e / cpu_baseline describing the same run. Also the multi-core leg of
the oracle on the batch (processes started together at a barrier), and the --shapes file that
lets a profiler run reuse the launch shapes of the plain run."""
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
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    for k in ("metric", "value", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["tol"] == 1e-10 and d["config"]["ntrace"] == 6400
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    sys.path.insert(0, repo_root)
    import bench
    assert d["config"] == bench.workload_config(bench.workload_spec("planar16"))
    assert "full solves" in d["cpu_baseline"]["sample"] and d["iterations"] > 0


def test_oracle_batch_leg_on_two_cores(repo_root):
    sys.path.insert(0, repo_root)
    import bench
    r = bench.oracle_batch_multicore(2)
    assert r["cores"] == 2 and r["all_ok"] and r["sample"] == ["C12xL50", "C32xL10"]
    assert r["value"] > 0 and r["wall_s"] > 0 and len(r["iterations"]) == 2
    assert all(i > 0 for i in r["iterations"])


class _ShapesStub:
    """Stands in for a Solver: records autotune and set_launch_shapes calls."""

    def __init__(self, tuned):
        self.tuned, self.calls, self.shapes = tuned, [], None

    def autotune(self):
        self.calls.append("autotune")
        self.shapes = self.tuned

    def launch_shapes(self):
        return self.shapes

    def set_launch_shapes(self, sweep, mg):
        self.calls.append("set")
        self.shapes = (tuple(sweep), [tuple(x) for x in mg])


def test_shapes_file_written_by_the_plain_run_and_applied_by_the_profiled_run(repo_root, tmp_path):
    """bench.py --shapes: the first run autotunes and writes its launch shapes; a second run of
    the same command applies them without tuning (so a profiler run times the same kernels);
    without the option every run autotunes."""
    sys.path.insert(0, repo_root)
    import bench
    tuned = ((32, 256), [(32, 256), (16, 128), (-1, 0)])
    path = str(tmp_path / "shapes.json")
    first = _ShapesStub(tuned)
    bench.tune_shapes(first, path)
    assert first.calls == ["autotune"] and os.path.exists(path)
    second = _ShapesStub(((1, 1), []))
    bench.tune_shapes(second, path)
    assert second.calls == ["set"] and second.launch_shapes() == tuned
    plain = _ShapesStub(tuned)
    bench.tune_shapes(plain, None)
    assert plain.calls == ["autotune"]
