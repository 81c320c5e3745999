"""bench.py --impl reference on the host (no GPU): the oracle arm prints one
JSON line with the main arm's metric, unit and direction, a config naming the
256x256 tile of the workload it times, and the cpu_baseline / e2e objects the
line format asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench

    assert line["impl"] == "reference"
    assert (line["metric"], line["unit"], line["higher_is_better"]) == (bench.METRIC, bench.UNIT, True)
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1
    cfg = line["config"]
    # the config states the tile the oracle actually times, not the full workload
    assert "256x256 tile" in cfg["workload"]
    assert cfg["queries_per_step"] == 482 and cfg["dictionary"] == 42802
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
