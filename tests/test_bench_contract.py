"""CPU checks of bench.py's measurement plumbing: the roofline peak comes from
the measured copy bandwidth, the committed ncu summary's DRAM traffic is used
only while the sweep sources it was taken on are unchanged, and the reference
arm (the FP64 oracle on the host cores) prints the JSON line the harness
reads."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_peak_is_the_measured_copy():
    peak, kind = bench.measured_peak_gbs()
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        assert peak == float(json.load(f)["hbm_gbs"]) and kind == "measured"


SUMMARIES = sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.startswith("k_sweep_plain_"))


@pytest.mark.parametrize("name", SUMMARIES)
def test_profiled_traffic_follows_the_source_hash(monkeypatch, name):
    path = os.path.join(ROOT, "profiles", name)
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: vals["source_hash"])
    assert bench.profiled_traffic(path) == float(vals["dram_bytes_per_launch_full_size"])
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic(path) is None


def test_reference_arm_prints_its_line():
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--workload", "settling_sphere"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    w, r, _, dist = bench.dist_setup()
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, 1.0 + r)  # each rank's own time; the job takes the slowest
    out.put((r, w, m, dist.get_backend()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    """The multi-rank plumbing of bench.py on two CPU ranks (gloo): both see
    world size 2 and the maximum of their times."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    assert all(w == 2 and m == 2.0 and b == "gloo" for _, w, m, b in res)


def test_reference_arm_under_torchrun_prints_once():
    """Launched like the harness launches N > 1 (torchrun, one process per
    rank), the reference arm runs on rank 0 alone and prints one line; the
    other rank exits 0 without work."""
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
