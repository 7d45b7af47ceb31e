"""bench.py's reference arm (the oracle timed on the host) keeps the benchmark's JSON contract.

The reference arm runs on the CPU, so its host logic is tested here: one JSON line from rank 0
with the GPU arm's metric, unit and config, the oracle as its cpu_baseline, an e2e equal to its
value with no copies, and nothing at all from the other ranks.
"""
import contextlib
import io
import json
import os
import subprocess
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"].startswith("stratified atmosphere 256^3")
    # ms_per_step is the measured time of one sample step (what the run spent); value is the
    # workload-size throughput, the sample scaled by the cell-count ratio 512
    assert d["value"] > 0 and abs(d["ms_per_step_at_workload_size"] - 2e3 / d["value"]) <= 1e-6 * d["ms_per_step"]
    assert abs(d["ms_per_step_at_workload_size"] - 512 * d["ms_per_step"]) <= 1e-6 * d["ms_per_step_at_workload_size"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert "32^3" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(steps=1, warmup=0, n=256, tol=1e-10, gpus=2)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args, 1)
    assert out.getvalue() == ""


def test_reference_arm_under_torchrun_two_ranks():
    # the launch the benchmark's N > 1 runs use, with gloo on the CPU: rank 0 prints one line,
    # rank 1 prints nothing, both exit 0 after the barrier
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--standalone", "--local-addr", "127.0.0.1",
                        "--nnodes=1", "--nproc-per-node", "2", os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
