"""bench.py --impl reference on the host (no GPU): one JSON line with the
keys the benchmark contract asks for, the same config dict as the GPU arm,
zero transfer bytes in e2e, and a cpu_baseline that describes the run.  The
small 8x8 TH P2/P1 workload keeps it to about a second."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "th_p2_8x8", "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] == line["value"]
    assert line["config"]["workload"] == "th_p2_8x8" and line["config"]["schedule"] == [2]
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    # the GPU arm builds its config with the same function and arguments
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    argv = sys.argv
    try:
        sys.argv = ["bench.py", "--workload", "th_p2_8x8"]
        a = bench.parse()
    finally:
        sys.argv = argv
    assert bench.step_config(a, W.workload("th_p2_8x8"), 1) == line["config"]
