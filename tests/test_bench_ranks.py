"""bench.py's multi-process launch on the CPU (gloo): with two ranks the
reference arm (the oracle) runs and prints on rank 0 only, the other rank
exits cleanly, and the JSON line carries the fields the benchmark contract
names.  The GPU arm is the same per-rank replica, so this covers the
rank/world logic without a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(900)
def test_reference_arm_two_ranks_gloo():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29517", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--oracle-workload", "cube4_k2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, env=env, timeout=850)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    for key in ("metric", "value", "unit", "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert key in line
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_bench_runs_name_existing_workloads():
    """Every workload of bench.py --configs (and --extra) is a named
    configuration, and the extra runs only use options bddc_setup takes."""
    import bench
    from synth.configs import CONFIGS
    runs = [r + ({},) for r in bench.CONFIG_RUNS] + list(bench.EXTRA_RUNS)
    for name, prec, theta, opt in runs:
        assert name in CONFIGS, name
        assert prec in (0, 1, 2) and theta >= 0.0
        assert set(opt) <= {"scaling", "reduced"}
        assert opt.get("scaling", 1) in (0, 1, 2)
