"""Benchmark of the lattice sweep (MLUPS and fraction of the HBM roofline).

Workload: one four-control-point metaball settling in a walled 128x128x256
D3Q19 lattice, BGK tau = 0.8, FP32 populations, 100 DEM sub-steps per LBM
step (the single non-spherical particle run, synthetic shape, seeded).  A
"step" is one whole LBM step through the C ABI: particle geometry and
binning, node classification with refilling, the fused sweep (plain bricks
and bricks near the particle, two kernels that run concurrently), the force
totals and the DEM sub-cycle.

Prints one JSON line.  value = lattice updates per second over all nodes of
all ranks (MLUPS); e2e = the same metric with the per-step host->device
particle upload and device->host force/state read through the public API;
roofline = the dominant kernel (the plain-brick sweep): its algorithmic bytes
(19 loads and 19 stores of every node it updates) over its CUDA-event time;
cpu_baseline = the FP64 CPU oracle timed on a bounded sample of the same
workload on the host cores.  The populations (2 x 319 MB) exceed the 129 MB
L2, so no flush is needed between steps.

--impl reference times the oracle itself (on rank 0; other ranks exit).
With torchrun and --gpus N > 1 every rank runs an independent replica on its
own GPU (the sweep does not exchange data), timed between barriers, max over
ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline per lattice sweep; drag rel. error vs FP64 oracle"
UNIT = "MLUPS"
BYTES_PER_VALUE = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}  # one stored population
# events around every 16th plain-sweep launch of the timed steps: the average
# launch duration from a sample, at a sixteenth of the events' cost
PLAIN_EVENT_EVERY = 16
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, the vendor's figure (the roofline's peak is the measured copy)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_sweep_plain_multi_particle_256x256x256.txt")
BRICK_NODES = 32 * 4 * 2
SWEEP_SOURCES = ["k_plain.cuh", "lbm_internal.cuh"]


WORKLOADS = ("multi_particle", "settling_metaball", "empty_box", "settling_sphere", "multi_particle_small",
             "batched_drag", "drag_gradient")
DEFAULT_WORKLOAD = "multi_particle"
DEFAULT_NAME = "multi_particle_200p_256x256x256"
# configurations reported beside a headline workload: (workload, storage, dem)
SECONDARY = {"multi_particle": (("multi_particle", "f16", "fp64"), ("multi_particle", "f32", "fp32"),
                                ("settling_metaball", "f32", "fp64"))}


def workload(name: str = DEFAULT_WORKLOAD, storage: str | None = None, dem: str | None = None):
    """The benchmark's workload (default) or a diagnostic one; storage
    overrides the workload's population storage."""
    wl = _workload(name)
    if dem:
        wl["dem"] = dem
    if storage:
        wl["storage"] = storage
        wl["name"] = f"{wl['name']}_{storage}" if storage != "f32" else wl["name"]
    if dem and dem != "fp64":
        wl["name"] = f"{wl['name']}_dem_{dem}"
    return wl


def _workload(name: str):
    from paper_2206_11634_gb300 import workloads
    if name == "settling_metaball":
        return workloads.settling_metaball(tau=0.8)
    if name == "empty_box":  # the same walled 128x128x256 lattice without a particle
        wl = workloads.empty_box(8, "f32", (0, 0, 0))
        wl.update(nx=128, ny=128, nz=256, name="empty_128x128x256")
        return wl
    if name == "settling_sphere":
        return workloads.settling_sphere()
    if name == "multi_particle":
        return workloads.multi_particle()
    if name == "multi_particle_small":  # the same particle density in 128x128x256 (profiling captures)
        return workloads.multi_particle(50, n=128, nz=256)
    if name == "batched_drag":  # the reference arm times its first case
        return workloads.batched_drag(64)[0]
    if name == "drag_gradient":  # the forward run of the gradient workload, as a lattice
        return gradient_lattice(workloads.adjoint_case())
    raise ValueError(name)


def gradient_lattice(case):
    """The drag-gradient case as a lattice workload: its fixed particle in the
    periodic box, started from the uniform flow u0 (the forward run)."""
    import numpy as np
    x = np.asarray(case["x"], dtype=np.float64)
    part = dict(cp=np.asarray(case["cp_world"]) - x, K=np.asarray(case["K"]), x=x, Rs=0.0, density=1.0,
                q=np.array([1.0, 0.0, 0.0, 0.0]), v=np.zeros(3), w=np.zeros(3), fixed=1, mass=1.0, inertia=np.eye(3))
    name = f"drag_gradient_{len(case['K'])}cp_{case['nx']}^3"
    return dict(name=name, nx=case["nx"], ny=case["ny"], nz=case["nz"], periodic=(1, 1, 1), tau=case["tau"],
                storage="f32", n_sub=0, gravity=(0.0, 0.0, 0.0), force=tuple(case["force"]), u0=tuple(case["u0"]),
                kn=0.0, eta_n=0.0, kt=0.0, eta_t=0.0, mu_s=0.0, c_tol=1e-6, particles=[part])


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def sweep_source_hash():
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2206_11634_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(path: str = PROFILE_SUMMARY):
    """DRAM bytes per sweep launch from the committed ncu summary, when it was
    taken on the current sweep source; else None."""
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != sweep_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.flush()
        rows = []
        for line in open(self.out.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_lattice(pkg, wl, stream):
    kw = dict(periodic=wl["periodic"], lattice=19, storage=wl["storage"], n_sub=wl["n_sub"],
              max_particles=max(1, len(wl["particles"])), tau=wl["tau"], gravity=wl["gravity"], force=wl["force"],
              kn=wl["kn"], eta_n=wl["eta_n"], kt=wl["kt"], eta_t=wl["eta_t"], mu_s=wl["mu_s"], c_tol=wl["c_tol"],
              dem_mode=pkg.DEM_MODE[wl.get("dem", "fp64")])
    lat = pkg.Lattice(wl["nx"], wl["ny"], wl["nz"], stream=stream, **kw)
    parts = []
    for p in wl["particles"]:
        kw = dict(q=p["q"], v=p["v"], w=p["w"], Rs=p["Rs"], density=p["density"], fixed=p["fixed"],
                  mass=p.get("mass", 0.0))
        if p.get("inertia") is not None:
            kw["inertia"] = p["inertia"]
        parts.append(pkg.make_particle(p["cp"], p["K"], p["x"], **kw))
    lat.set_particles(parts)
    return lat


def oracle_sample(wl, steps: int, nthreads: int = 0):
    """Time `steps` steps of the FP64 oracle on the full workload (nthreads
    OpenMP threads; 0: all)."""
    import oracle
    o = oracle.Oracle(wl["nx"], wl["ny"], wl["nz"], Q=19, periodic=tuple(wl["periodic"]), tau=wl["tau"],
                      n_sub=wl["n_sub"], gravity=wl["gravity"], force=wl["force"], kn=wl["kn"], eta_n=wl["eta_n"],
                      kt=wl["kt"], eta_t=wl["eta_t"], mu_s=wl["mu_s"], c_tol=wl["c_tol"],
                      u0=tuple(wl.get("u0", (0.0, 0.0, 0.0))), nthreads=nthreads)
    o.set_particles([oracle.make_particle(p["cp"], p["K"], p["x"], q=p["q"], v=p["v"], w=p["w"], Rs=p["Rs"],
                                          density=p["density"], fixed=p["fixed"]) for p in wl["particles"]])
    o.step(1)  # first step pays the page-in of the arrays
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    n = wl["nx"] * wl["ny"] * wl["nz"]
    return n * steps / dt / 1e6, dt


DRAG_REFERENCE = os.path.join(ROOT, "tests", "golden", "drag_reference.json")


def drag_check(pkg, storage: str):
    """Relative error of the drag F_x of the drag case (a fixed metaball in a
    periodic, body-force-driven 48^3 box, 1000 steps) in this storage form,
    against the FP64 oracle's value stored in tests/golden/drag_reference.json
    (written by tests/golden/make_drag_reference.py)."""
    import numpy as np
    from paper_2206_11634_gb300 import workloads
    ref = json.load(open(DRAG_REFERENCE))
    wl = workloads.drag_case(storage)
    wl["particles"][0]["x"] = np.array(ref["x"])
    lat = make_lattice(pkg, wl, None)
    lat.step(ref["steps"])
    F, _ = lat.forces()
    return {"rel_error_Fx": float(f"{abs(F[0, 0] - ref['F'][0]) / abs(ref['F'][0]):.3e}"), "case": ref["case"],
            "steps": ref["steps"], "storage": storage, "reference": "FP64 oracle, tests/golden/drag_reference.json"}


def omp_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


# the reference arm times the oracle on at most this much of the requested
# steps (the 256^3 workload takes about half a second per step on 16 cores)
REFERENCE_MAX_SECONDS = 60.0
REFERENCE_MAX_WARMUP = 2


def run_reference(args):
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return 0
    wl = workload(args.workload)
    import oracle
    oracle.build()
    warm = max(1, min(args.warmup, REFERENCE_MAX_WARMUP))
    _, t_warm = oracle_sample(wl, warm)
    per_step = t_warm / warm
    steps = max(1, min(args.steps, int(REFERENCE_MAX_SECONDS / max(per_step, 1e-6))))
    mlups, dt = oracle_sample(wl, steps)
    cores = omp_threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": round(dt / steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "lattice": "D3Q19", "storage": "f64", "tau": wl["tau"],
                       "n_sub": wl["n_sub"], "particles": len(wl["particles"])},
            "cpu_baseline": {"value": round(mlups, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} of the {args.steps} requested steps of the full "
                                       f"{wl['nx']}x{wl['ny']}x{wl['nz']} workload, {dt:.1f} s"},
            "e2e": {"value": round(mlups, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(lat, stream, dist, steps: int, min_seconds: float, max_repeats: int = 200):
    """Time `steps` steps between barriers and device synchronisation, with
    CUDA events on the lattice's stream, repeated until `min_seconds` have
    elapsed (at least once); returns the per-repeat milliseconds."""
    import torch
    out = []
    t0 = time.perf_counter()
    while not out or (time.perf_counter() - t0 < min_seconds and len(out) < max_repeats):
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        start.record(stream)
        lat.step(steps)
        stop.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
        out.append(start.elapsed_time(stop))
    return out


def dem_label(wl):
    storage, dem = wl["storage"], wl.get("dem", "fp64")
    if storage == "f64" or dem == "fp64_all":
        return "FP64 rigid-body integrator and contact geometry"
    if dem == "fp32":
        return "compensated-FP32 rigid-body integrator, FP32 contact geometry"
    return "FP64 rigid-body integrator, FP32 contact geometry"


def plain_roofline(lat, wl, plain_ms, plain_n, peak):
    """Achieved HBM bandwidth of the plain sweep: the survey's algorithmic
    bytes per lattice update (19 loads + 19 stores of the stored population
    type, plus the 2-byte node flag) times the nodes one launch updates (every
    node outside the near bricks), over its mean CUDA-event duration."""
    nodes = wl["nx"] * wl["ny"] * wl["nz"]
    near_bricks = lat.counters()["near_bricks"]
    plain_nodes = max(0, nodes - near_bricks * BRICK_NODES)
    per_lu = 2 * 19 * BYTES_PER_VALUE[wl["storage"]] + 2
    alg = per_lu * plain_nodes
    avg_s = plain_ms / max(1, plain_n) * 1e-3
    achieved = alg / avg_s / 1e9 if avg_s > 0 else 0.0
    return dict(achieved=achieved, frac=achieved / peak, bytes=alg, per_lu=per_lu, plain_nodes=plain_nodes,
                avg_us=avg_s * 1e6)


def measure_workload(pkg, wl, args, dist, local, min_seconds, stream=None):
    """Warm-up, then the timed region (K steps, repeated to min_seconds, the
    median kept), events around every PLAIN_EVENT_EVERY-th plain-sweep
    launch of the timed steps (their mean is the roofline's duration)."""
    import torch
    stream = stream or torch.cuda.Stream()
    lat = make_lattice(pkg, wl, stream)
    lat.step(max(3, args.warmup))
    torch.cuda.synchronize()
    lat.profile(True, kernels=["k_sweep_plain"], every=PLAIN_EVENT_EVERY)
    with ClockSampler(local) as clocks:
        reps = timed_steps(lat, stream, dist, args.steps, min_seconds)
    prof_timed = lat.profile_read()
    lat.profile(False)
    lat.check()
    ms = max_over_ranks(dist, statistics.median(reps))
    return lat, stream, reps, ms, prof_timed, clocks.summary()


def run_gpu(args):
    import torch

    world, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    import paper_2206_11634_gb300 as pkg
    from paper_2206_11634_gb300 import build as lib_build
    if rank == 0 or not os.path.exists(pkg.LIB_PATH):
        lib_build.build()
    barrier(dist)
    wl = workload(args.workload, args.storage, args.dem)
    nodes = wl["nx"] * wl["ny"] * wl["nz"]
    peak, peak_kind = measured_peak_gbs()

    lat, stream, reps, ms, prof_timed, clocks = measure_workload(pkg, wl, args, dist, local, args.min_seconds)
    fl = lat.flags()
    n_fluid = int((fl == 0).sum().item())
    kps = lat.kernels_per_step()
    value = world * nodes * args.steps / (ms * 1e-3) / 1e6
    ms_step = ms / args.steps
    plain_ms, plain_n = prof_timed["k_sweep_plain"]
    rf = plain_roofline(lat, wl, plain_ms, plain_n, peak)
    # the per-kernel breakdown from a separate pass with events around every
    # kernel (they lengthen the step)
    prof_steps = min(args.steps, 200)
    lat.profile(True)
    lat.step(prof_steps)
    prof = lat.profile_read()
    lat.profile(False)
    lat.check()

    # end-to-end through the public API with host buffers: per step upload
    # the particle state, step, read back forces, torques and state
    np_ = len(wl["particles"])
    state = (pkg.LbmParticle * max(1, np_))()
    import numpy as np
    F = np.zeros((max(1, np_), 3))
    T = np.zeros((max(1, np_), 3))
    import ctypes as C
    L = lat.L
    L.lbm_get_forces(lat.h, None, None, state)
    e2e_steps = max(4, args.steps // 4)
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = L.lbm_set_particles(lat.h, state, np_)
        rc |= L.lbm_step(lat.h, 1)
        rc |= L.lbm_get_forces(lat.h, F.ctypes.data_as(C.POINTER(C.c_double)),
                               T.ctypes.data_as(C.POINTER(C.c_double)), state)
        if rc:
            raise RuntimeError(L.lbm_last_error(lat.h).decode())
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    barrier(dist)
    e2e_value = world * nodes * e2e_steps / e2e_s / 1e6
    h2d = C.sizeof(pkg.LbmParticle) * np_
    d2h = 48 * np_ + C.sizeof(pkg.LbmParticle) * np_
    del lat
    torch.cuda.synchronize()

    # further configurations, reported beside the headline (not the value)
    secondary = []
    if not args.no_secondary:
        for name, storage, dem in SECONDARY.get(args.workload, ()):
            w2 = workload(name, storage, dem)
            n2 = w2["nx"] * w2["ny"] * w2["nz"]
            lat2, _, reps2, ms2, pt2, ck2 = measure_workload(pkg, w2, args, dist, local, 0.5)
            r2 = plain_roofline(lat2, w2, *pt2["k_sweep_plain"], peak)
            secondary.append({"workload": w2["name"], "storage": w2["storage"], "dem": dem_label(w2),
                              "value": round(world * n2 * args.steps / (ms2 * 1e-3) / 1e6, 2), "unit": UNIT,
                              "ms_per_step": round(ms2 / args.steps, 4), "timed_repeats": len(reps2),
                              "plain_sweep_frac": round(r2["frac"], 4), "plain_sweep_us": round(r2["avg_us"], 2),
                              "clocks_sm_mhz": ck2.get("sm_mhz")})
            del lat2
            torch.cuda.synchronize()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # the committed capture is of the default workload's plain sweep
    traffic = profiled_traffic() if (wl["name"], wl["storage"]) == (DEFAULT_NAME, "f32") else None
    kernels = {k: {"avg_us": round(v[0] / max(1, v[1]) * 1e3, 3), "launches": v[1],
                   "share": round(v[0] / max(1e-12, sum(x[0] for x in prof.values())), 4)}
               for k, v in prof.items() if v[1] > 0}

    # CPU baseline: the oracle as it stands on this host, bounded sample
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu_steps = args.cpu_steps or max(1, int(round(4e8 / nodes)))
        mlups, dt = oracle_sample(wl, cpu_steps)
        cpu = {"value": round(mlups, 4), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": f"{cpu_steps} steps of the full {wl['nx']}x{wl['ny']}x{wl['nz']} workload, FP64, "
                         f"{dt:.1f} s"}
        one_steps = max(1, cpu_steps // 20)
        mlups1, dt1 = oracle_sample(wl, one_steps, nthreads=1)
        cpu["one_core"] = {"value": round(mlups1, 4), "unit": UNIT, "cores": 1,
                           "sample": f"{one_steps} steps, {dt1:.1f} s"}

    pop_mb = 19 * BYTES_PER_VALUE[wl["storage"]] * nodes / 1e6
    l2_note = (f"no flush: populations 2x{pop_mb:.0f} MB exceed the 129 MB L2" if pop_mb > 129 else
               f"populations 2x{pop_mb:.0f} MB fit the 129 MB L2 (no flush; L2-resident)")
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl["storage"], "data": "synthetic",
            "config": {"workload": wl["name"], "lattice": "D3Q19", "storage": wl["storage"], "tau": wl["tau"],
                       "n_sub": wl["n_sub"], "particles": len(wl["particles"]), "nodes": nodes,
                       "fluid_nodes": n_fluid, "dem": dem_label(wl), "l2": l2_note,
                       "timing": f"the {args.steps} steps timed {len(reps)} times (at least "
                                 f"{args.min_seconds:g} s in all); median of "
                                 f"{[round(r, 3) for r in sorted(reps)[:3]]}.. ms",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "roofline": {"bound": "hbm", "achieved": round(rf["achieved"], 1), "peak": peak, "unit": "GB/s",
                         "frac": round(rf["frac"], 4), "traffic": traffic, "peak_kind": f"{peak_kind} copy",
                         "frac_of_nominal": round(rf["achieved"] / NOMINAL_HBM_GBS, 4),
                         "nominal_peak": NOMINAL_HBM_GBS, "kernel": "k_sweep_plain",
                         "bytes_per_launch": rf["bytes"],
                         "bytes_per_lattice_update": rf["per_lu"], "plain_nodes": rf["plain_nodes"],
                         "avg_launch_us": round(rf["avg_us"], 3),
                         "avg_launch_le_step": rf["avg_us"] <= ms_step * 1e3,
                         "timed_launches_sampled": f"{plain_n} (every {PLAIN_EVENT_EVERY}th plain-sweep launch of "
                                                   f"all {len(reps) * args.steps} timed steps)"},
            "kernels": kernels,
            "kernels_note": f"per-kernel events around every launch, separate pass of {prof_steps} steps",
            "gpu_launches": kps * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "secondary": secondary,
            "drag": drag_check(pkg, wl["storage"])}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Workload 5: 64 independent periodic drag cases, sides 48..128, one
    fixed metaball each, stepped as a batch (one launch per kernel for all
    cases, replayed CUDA graphs; the fixed geometry is recorded once and every
    later step is the link and plain kernels of the fixed-geometry sweep)
    after the autotuner picked the schedule.  value = aggregate MLUPS over all
    cases."""
    import torch
    import numpy as np

    world, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    import paper_2206_11634_gb300 as pkg
    from paper_2206_11634_gb300 import build as lib_build, workloads
    if rank == 0 or not os.path.exists(pkg.LIB_PATH):
        lib_build.build()
    barrier(dist)
    storage = args.storage or "f32"
    cases = workloads.batched_drag(64, storage)
    nodes = sum(c["nx"] * c["ny"] * c["nz"] for c in cases)
    kws = []
    for c in cases:
        kw = dict(nx=c["nx"], ny=c["ny"], nz=c["nz"], periodic=c["periodic"], lattice=19, storage=storage,
                  n_sub=0, max_particles=1, tau=c["tau"], force=c["force"])
        kws.append(kw)
    stream = torch.cuda.Stream()
    bt = pkg.Batch(kws, stream=stream)
    for k, c in enumerate(cases):
        p = c["particles"][0]
        bt.set_particles(k, [pkg.make_particle(p["cp"], p["K"], p["x"], q=p["q"], fixed=1, mass=p["mass"],
                                               inertia=p["inertia"])])
    g, chunk, tune_ms = bt.tune(2)
    bt.step(max(3, args.warmup))
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier(dist)
        torch.cuda.synchronize()
        start.record(stream)
        bt.step(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
    ms = max_over_ranks(dist, start.elapsed_time(stop))
    value = world * nodes * args.steps / (ms * 1e-3) / 1e6
    # end to end: per call of one step, read back every case's drag
    e2e_steps = max(1, args.steps // 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        bt.step(1)
        bt.all_forces()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    e2e_value = world * nodes * e2e_steps / e2e_s / 1e6
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = measured_peak_gbs()
    alg = 2 * 19 * BYTES_PER_VALUE[storage] * nodes
    achieved = alg / (ms / args.steps * 1e-3) / 1e9
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        c0 = dict(cases[0])
        c0["n_sub"] = 0
        cpu_steps = max(1, (args.cpu_steps or 200) // 2)
        mlups, dt = oracle_sample(c0, cpu_steps)
        cpu = {"value": round(mlups, 4), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": f"{cpu_steps} steps of case 0 ({c0['nx']}x{c0['ny']}x{c0['nz']}), FP64, {dt:.1f} s; "
                         f"the oracle steps the cases one after another"}
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": storage, "data": "synthetic",
            "config": {"workload": f"batched_drag_64cases_{storage}", "lattice": "D3Q19", "storage": storage,
                       "cases": len(cases), "nodes": nodes, "sides": "48..128", "tau": 0.8,
                       "schedule": {"chain_ctas_per_case": g, "plain_blocks_per_cta": chunk,
                                    "tuned_ms_per_step": round(tune_ms, 4)},
                       "l2": "no flush: populations exceed the 129 MB L2", "parallelism": f"replicas x{world}"},
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 48 * len(cases), "steps": e2e_steps},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": f"{peak_kind} copy",
                         "kernel": "whole batched step (all phases, all cases)", "bytes_per_launch": alg},
            # the fixed-geometry sweep's link and plain kernels (the particles
            # are fixed: binning, flag pass and brick sweeps ran only in the
            # first steps, before the timed region)
            "gpu_launches": 2 * args.steps,
            "clocks": clocks.summary(), "cpu_baseline": cpu, "drag": drag_check(pkg, storage)}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# gradient evaluations timed per run (each is a 500-step forward run plus its
# adjoint, ~0.2 s): the requested step count is capped at this
GRADIENT_MAX = 8


def run_gradient(args):
    """Workload 4: d(mean drag)/d(control points, weights) of one fixed
    six-control-point metaball in a periodic 96^3 box, T = 500 steps, window
    W = 100, through the library's hand-written adjoint (flags frozen, sqrt(T)
    checkpoints).  A "step" here is one gradient evaluation (forward run and
    backward run); value = lattice updates of the objective (N x T per
    gradient) per second of forward plus backward time."""
    import torch
    import numpy as np

    world, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    import paper_2206_11634_gb300 as pkg
    from paper_2206_11634_gb300 import build as lib_build, workloads
    if rank == 0 or not os.path.exists(pkg.LIB_PATH):
        lib_build.build()
    barrier(dist)
    from paper_2206_11634_gb300.adjoint import AdjointDrag
    case = workloads.adjoint_case()
    x = np.asarray(case["x"], dtype=np.float64)
    part = pkg.make_particle(np.asarray(case["cp_world"]) - x, case["K"], x, q=(1.0, 0.0, 0.0, 0.0), fixed=1,
                             mass=1.0, inertia=np.eye(3))
    stream = torch.cuda.Stream()
    eng = AdjointDrag(case["nx"], case["ny"], case["nz"], particle=part, T=case["T"], W=case["W"], tau=case["tau"],
                      u0=case["u0"], force=case["force"], stream=stream)
    nodes = case["nx"] * case["ny"] * case["nz"]
    grads = max(1, min(args.steps, GRADIENT_MAX))
    warm = max(1, min(args.warmup, 2))
    cp, K = case["cp_world"], case["K"]
    for _ in range(warm):
        eng.forward_np(cp, K)
        eng.backward_np()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ms_f = ms_b = 0.0
    with ClockSampler(local) as clocks:
        barrier(dist)
        torch.cuda.synchronize()
        for _ in range(grads):
            ev[0].record(stream)
            eng.forward_np(cp, K)
            ev[1].record(stream)
            g_cp, g_K = eng.backward_np()
            ev[2].record(stream)
            torch.cuda.synchronize()
            ms_f += ev[0].elapsed_time(ev[1])
            ms_b += ev[1].elapsed_time(ev[2])
        barrier(dist)
    ms = max_over_ranks(dist, ms_f + ms_b)
    T = case["T"]
    value = world * nodes * T * grads / (ms * 1e-3) / 1e6
    # end to end: the autograd function from host tensors to host gradients
    e2e_grads = max(1, grads // 2)
    cpt = torch.tensor(cp, dtype=torch.float64, requires_grad=True)
    Kt = torch.tensor(K, dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_grads):
        cpt.grad = None
        Kt.grad = None
        J = eng(cpt, Kt)
        J.backward()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    e2e_value = world * nodes * T * e2e_grads / e2e_s / 1e6
    ncp = len(K)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    # the forward step kernel: 19 loads and 19 stores of FP32 per node and step
    peak, peak_kind = measured_peak_gbs()
    step_s = ms_f / grads / T * 1e-3
    alg = 2 * 19 * 4 * nodes
    achieved = alg / step_s / 1e9
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu_steps = max(1, (args.cpu_steps or 200) // 2)
        mlups, dt = oracle_sample(gradient_lattice(case), cpu_steps)
        cpu = {"value": round(mlups, 4), "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": f"{cpu_steps} forward steps of the {case['nx']}^3 case, FP64, {dt:.1f} s (the oracle has "
                         f"no adjoint: its gradient by central differences takes {2 * 4 * ncp} such runs)"}
    info = eng.info()
    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": grads,
            "warmup": warm, "ms_per_step": round(ms / grads, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"drag_gradient_{ncp}cp_{case['nx']}^3", "lattice": "D3Q19", "storage": "f32",
                       "T": T, "W": case["W"], "tau": case["tau"], "links": info["nlinks"],
                       "checkpoint_every": info["checkpoint_every"], "step": "one gradient (forward + backward)",
                       "forward_ms": round(ms_f / grads, 3), "backward_ms": round(ms_b / grads, 3),
                       "l2": "no flush: two FP32 population arrays of 67 MB each, about the 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": 32 * ncp,
                    "d2h_bytes_per_step": 8 + 32 * ncp, "steps": e2e_grads},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": f"{peak_kind} copy",
                         "kernel": "forward step (k_adj_step)", "bytes_per_launch": alg,
                         "avg_launch_us": round(step_s * 1e6, 3)},
            "gradient": {"dJ_dK": [float(f"{v:.6e}") for v in g_K]},
            # per gradient: q and the initial state, T forward steps; T - C
            # recomputed steps (C checkpoints), three adjoint kernels per step
            # and the chain rule to the shape
            "gpu_launches": grads * (2 + T + (T - -(-T // info["checkpoint_every"])) + 3 * T + 1),
            "clocks": clocks.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--min-seconds", type=float, default=1.0,
                    help="repeat the timed steps until this much time has passed (median reported)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the configurations reported beside the headline")
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--cpu-steps", type=int, default=None,
                    help="oracle steps of the CPU baseline (default: about 4e8 lattice updates)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16", "f64"], default=None,
                    help="population storage (default: the workload's own)")
    ap.add_argument("--dem", choices=["fp64", "fp32", "fp64_all"], default=None,
                    help="DEM arithmetic: fp64 (default) the FP64 rigid-body integrator, FP32 contact geometry "
                         "below FP64 storage; fp32 the compensated-FP32 integrator; fp64_all FP64 contact geometry too")
    ap.add_argument("--workload", choices=WORKLOADS, default=DEFAULT_WORKLOAD,
                    help="diagnostic workloads besides the default benchmark workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_drag":
        return run_batch(args)
    if args.workload == "drag_gradient":
        return run_gradient(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
