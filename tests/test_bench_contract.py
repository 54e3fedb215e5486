"""CPU checks of bench.py's measurement plumbing: the roofline peak comes from
the measured copy bandwidth, the committed ncu summary's DRAM traffic is used
only while the sweep sources it was taken on are unchanged, and the reference
arm (the FP64 oracle on the host cores) prints the JSON line the harness
reads."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_peak_is_the_measured_copy():
    peak, kind = bench.measured_peak_gbs()
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        assert peak == float(json.load(f)["hbm_gbs"]) and kind == "measured"


def test_profiled_traffic_follows_the_source_hash(monkeypatch):
    vals = {}
    for line in open(bench.PROFILE_SUMMARY):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: vals["source_hash"])
    assert bench.profiled_traffic() == float(vals["dram_bytes_per_launch_full_size"])
    # the summary's traffic is the sum of its read and write bytes
    assert float(vals["dram_bytes_per_launch_full_size"]) == float(vals["dram_bytes_read"]) + float(
        vals["dram_bytes_write"])
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic() is None


def test_reference_arm_prints_its_line():
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
