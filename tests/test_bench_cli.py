"""bench.py's reference arm (the oracle on the host cores) prints one JSON line with
the benchmark's metric and workload; run here on a small sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    proc = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--cpu-scale", "11"], cwd=ROOT, capture_output=True, text=True,
                          timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    lines = [l for l in proc.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "triangles surveyed/s" and d["unit"] == "triangles/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "R-MAT scale 24" in d["config"]["workload"]


def test_cpu_baseline_reports_all_cores_and_one_thread():
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    d = bench.cpu_baseline(argparse.Namespace(cpu_scale=12))
    assert d["kind"] == "oracle" and d["cores"] == (os.cpu_count() or 1) and d["value"] > 0
    assert d["single_thread"]["cores"] == 1 and d["single_thread"]["value"] > 0
    assert "scale 12" in d["sample"] and "scale 10" in d["single_thread"]["sample"]
    assert isinstance(d["cpu_model"], str)


def test_compulsory_bytes_are_part_of_the_algorithmic_bytes():
    sys.path.insert(0, ROOT)
    import bench
    st = {"num_vertices": 1000, "num_edges": 5000}
    assert bench.compulsory_bytes(st) == 9 * 1000 + 26 * 5000
    assert bench.algorithmic_bytes(st, 0, 0) == bench.compulsory_bytes(st)
    assert bench.algorithmic_bytes(st, 7, 3) == bench.compulsory_bytes(st) + 4 * 7 + 5 * 3
