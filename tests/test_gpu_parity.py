"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (element by element, stated per test):
- node flags: bit-exact (inputs rejected when a node lies within 1e-9
  relative of a surface);
- one step, FP64 storage: populations within 1e-13 absolute (values ~0.1;
  only the rounding order differs), force/torque within 1e-11 of the
  force scale;
- one step, FP32 storage: populations within 2e-6 absolute -- the collision
  of ~0.1-sized values in FP32 rounds at ~1e-8 per operation, and the link
  fraction q of Eq. (27) is computed from FP32 metaball values (relative error
  <= 2^-13, which moves a VIBB population by at most ~1e-6); forces within
  2e-6 per boundary link plus 1e-5 relative;
- FP16 / BF16 offset storage: the stored offset s = f/w - rho0 is rounded to
  11 / 8 significant bits, so a population carries an absolute error of at
  most w |s| 2^-11 (resp. 2^-8) on top of the FP32 error: 2e-5 / 1.5e-4.
"""
import numpy as np
import pytest

from tests import _helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def pkg():
    from paper_2206_11634_gb300 import build as b
    b.build()
    import paper_2206_11634_gb300 as p
    return p


@pytest.fixture(scope="module")
def W():
    from paper_2206_11634_gb300 import workloads
    return workloads


POP_TOL = {"f64": 1e-13, "f32": 2e-6, "f16": 2e-5, "bf16": 1.5e-4}


def _sync_populations(gpu, orc, rng, amp=1e-2):
    """Random populations into the GPU (in its storage format), read back as
    FP64, injected identically into the oracle."""
    f = rng.uniform(1 - amp, 1 + amp, (gpu.Q,) + gpu.shape) * orc.w[:, None, None, None]
    gpu.set_populations(torch.from_numpy(f).cuda())
    back = gpu.populations().cpu().numpy()
    orc.set_populations(back)
    return back


def _compare_step(pkg, oracle_mod, wl, storage, Q=19, rng_seed=0, steps=1, amp=1e-2, check_forces=True, **over):
    rng = np.random.default_rng(rng_seed)
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl, Q=Q, storage=storage, **over)
    orc = H.make_oracle(oracle_mod, wl, Q=Q, **over)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    _sync_populations(gpu, orc, rng, amp)
    gpu.step(steps)
    orc.step(steps)
    fl = gpu.flags().cpu().numpy()
    own = orc.owner()
    assert np.array_equal(fl - 1, own), "flags differ"
    fluid = own < 0
    fg = gpu.populations().cpu().numpy()
    fo = orc.populations()
    err = np.abs(fg - fo)[:, fluid].max() if fluid.any() else 0.0
    tol = POP_TOL[storage] * (3 if steps > 1 else 1)
    assert err <= tol, f"population error {err:.3e} > {tol:.1e}"
    out = dict(gpu=gpu, orc=orc, err=err)
    if check_forces and wl["particles"]:
        Fg, Tg = gpu.forces()
        Fo, To = orc.forces()
        nl = max(1, orc.counters()["nlinks"])
        assert gpu.counters()["nlinks"] == orc.counters()["nlinks"]
        if storage == "f64":
            ftol = 1e-11 * nl * 0.2
        else:
            ftol = POP_TOL[storage] * nl + 1e-5 * max(np.abs(Fo).max(), 1e-3)
        assert np.abs(Fg - Fo).max() <= ftol, (Fg, Fo)
        # torque lever arms are O(radius)
        assert np.abs(Tg - To).max() <= 20 * ftol, (Tg, To)
        out.update(F=(Fg, Fo), T=(Tg, To))
    return out


# --------------------------------------------------------------------------
# workloads for the one-step comparisons
# --------------------------------------------------------------------------
def wl_periodic_empty(W):
    wl = W.empty_box(24, "f32", (1, 1, 1))
    wl.update(nx=24, ny=20, nz=16)
    return wl


def wl_walls_guo_ragged(W):
    wl = W.empty_box(8, "f32", (0, 1, 0))
    wl.update(nx=45, ny=13, nz=9, force=(2e-5, -1e-5, 3e-5), tau=0.62)
    return wl


def wl_metaball(W, periodic=(0, 0, 0), n=(40, 36, 44)):
    rng = np.random.default_rng(11)
    cp, K = W.random_metaball(rng, 4, 4.0)
    wl = W.empty_box(8, "f32", periodic)
    wl.update(nx=n[0], ny=n[1], nz=n[2], tau=0.8)
    wl["particles"] = [W._particle(cp, K, (n[0] / 2 - 0.3, n[1] / 2 + 0.2, n[2] / 2 + 0.1),
                                   q=(0.8, 0.3, -0.4, 0.33), v=(0.01, -0.02, 0.015), w=(0.002, -0.001, 0.003),
                                   density=1.2, fixed=1)]
    return H.fixed_mass(wl)


def wl_touching(W):
    """A sphere touching the bottom wall and two overlapping metaballs: the
    missing force points of §2.3.5 item 2 are exercised."""
    wl = W.empty_box(8, "f32", (1, 1, 0))
    wl.update(nx=36, ny=28, nz=24, tau=0.9)
    wl["particles"] = [
        W._particle([[0, 0, 0]], [16.0], (9.3, 10.1, 3.2), fixed=1, v=(0.01, 0, 0), w=(0, 0.004, 0)),
        W._particle([[0, 0, 0], [1, 0.5, 0]], [9.0, 7.0], (20.3, 12.1, 11.6), fixed=1, v=(0, 0.01, 0)),
        W._particle([[0, 0, 0]], [12.0], (26.2, 12.4, 12.2), fixed=1, w=(0.002, 0, 0.001)),
    ]
    return H.fixed_mass(wl)


def wl_multi(W, n=64, nz=64, count=10):
    wl = W.multi_particle(count, n=n, nz=nz, storage="f32", steps=4, seed_offset=7)
    for p in wl["particles"]:
        p["fixed"] = 1
        p["v"] = np.array([0.005, -0.004, 0.006])
    return H.fixed_mass(wl)


def wl_wrap(W):
    """A metaball straddling the periodic x and y faces."""
    rng = np.random.default_rng(5)
    cp, K = W.random_metaball(rng, 3, 3.0)
    wl = W.empty_box(8, "f32", (1, 1, 0))
    wl.update(nx=32, ny=24, nz=20)
    wl["particles"] = [W._particle(cp, K, (0.4, 23.3, 9.8), q=(0.6, 0.2, 0.7, 0.33), v=(0.01, 0.0, -0.01),
                                   fixed=1)]
    return H.fixed_mass(wl)


CASES = ["periodic_empty", "walls_guo_ragged", "metaball", "touching", "multi", "wrap"]


def _case(W, name):
    return {"periodic_empty": wl_periodic_empty, "walls_guo_ragged": wl_walls_guo_ragged, "metaball": wl_metaball,
            "touching": wl_touching, "multi": wl_multi, "wrap": wl_wrap}[name](W)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["metaball", "touching", "multi", "wrap"])
def test_flags_bit_exact(pkg, oracle_mod, W, case):
    wl = H.with_margin(oracle_mod, _case(W, case))
    gpu = H.make_gpu(pkg, wl, n_sub=0)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    gpu.step(1)
    o = H.make_oracle(oracle_mod, wl)
    o.set_particles(H.oracle_particles(oracle_mod, wl))
    own = o.classify()
    fl = gpu.flags().cpu().numpy()
    assert (own >= 0).sum() > 50
    assert np.array_equal(fl - 1, own)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES)
def test_one_step(pkg, oracle_mod, W, case, storage):
    _compare_step(pkg, oracle_mod, _case(W, case), storage)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case", ["walls_guo_ragged", "metaball", "touching"])
def test_one_step_d3q15(pkg, oracle_mod, W, case, storage):
    _compare_step(pkg, oracle_mod, _case(W, case), storage, Q=15)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case", ["metaball", "touching", "wrap"])
def test_one_step_exact_q(pkg, oracle_mod, W, case, storage):
    """Link fraction by Newton's method on Eq. (26) (option q_exact, §2.3.1)
    on both sides, for the links of Eq. (28) and the missing force points.
    The tolerances stay those of Eq. (27): the FP64 iterations follow the
    oracle's; in FP32 the root is found to the residual's rounding, a q error
    of a few 1e-7 that moves an unknown by ~1e-8.  The option must change the
    result: the forces differ from the Eq. (27) run by far more than the
    tolerance."""
    ex = _compare_step(pkg, oracle_mod, _case(W, case), storage, q_exact=1)
    lin = _compare_step(pkg, oracle_mod, _case(W, case), storage, q_exact=0)
    Fe, Fl = ex["F"][0], lin["F"][0]
    assert np.abs(Fe - Fl).max() > 1e-4 * np.abs(Fl).max(), (Fe, Fl)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["wall", "pair"])
def test_missing_force_points_ab(pkg, oracle_mod, W, storage, kind):
    """§2.3.5 item 2 as an A/B comparison (the two-sphere test of §3.3, at
    rest): particles resting against a wall or against each other in fluid
    at rest.  With the missing force points the force and torque are exactly
    zero (every crossing link is counted once, and in offset form each term
    is zero at rest), without them the links hidden by the contact leave a
    net force of order 0.1, equal to the oracle's within the one-step force
    tolerance."""
    wl = W.empty_box(8, storage, (1, 1, 0) if kind == "wall" else (1, 1, 1))
    if kind == "wall":
        wl.update(nx=20, ny=20, nz=20)
        wl["particles"] = [W._particle([[0, 0, 0]], [16.0], (9.3, 10.1, 3.2), fixed=1)]
    else:
        wl.update(nx=24, ny=24, nz=24)
        wl["particles"] = [W._particle([[0, 0, 0], [1, 0.5, 0]], [9.0, 7.0], (8.3, 12.1, 11.6), fixed=1),
                           W._particle([[0, 0, 0]], [12.0], (14.2, 12.4, 12.2), fixed=1)]
    wl = H.with_margin(oracle_mod, H.fixed_mass(wl, mass=1.0, inertia=1.0))
    out = {}
    for mf in (1, 0):
        gpu = H.make_gpu(pkg, wl, missing_force=mf)
        orc = H.make_oracle(oracle_mod, wl, missing_force=mf)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        orc.set_particles(H.oracle_particles(oracle_mod, wl))
        gpu.step(3)
        orc.step(3)
        assert np.array_equal(gpu.flags().cpu().numpy() - 1, orc.owner())
        out[mf] = (gpu.forces(), orc.forces(), orc.counters()["nlinks"])
    (Fg, Tg), _, _ = out[1]
    assert np.abs(Fg).max() <= 1e-12 and np.abs(Tg).max() <= 1e-12, (Fg, Tg)
    (Fg, Tg), (Fo, To), nl = out[0]
    assert np.abs(Fo).max() > 0.1
    ftol = 1e-11 * nl * 0.2 if storage == "f64" else POP_TOL[storage] * nl + 1e-5 * np.abs(Fo).max()
    assert np.abs(Fg - Fo).max() <= ftol, (Fg, Fo)
    assert np.abs(Tg - To).max() <= 20 * ftol, (Tg, To)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("case", ["metaball", "touching"])
def test_one_step_reduced_storage(pkg, oracle_mod, W, case, storage):
    _compare_step(pkg, oracle_mod, _case(W, case), storage)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_three_steps_moving_geometry(pkg, oracle_mod, W, storage):
    """Particles that move between steps (DEM off, positions set by hand):
    new fluid nodes are refilled (§2.3.3) on both sides."""
    wl = wl_metaball(W, periodic=(1, 1, 1), n=(36, 36, 36))
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl, storage=storage)
    orc = H.make_oracle(oracle_mod, wl)
    rng = np.random.default_rng(3)
    refilled = 0
    p0 = wl["particles"][0]
    for k in range(3):
        p0["x"] = p0["x"] + np.array([0.37, -0.29, 0.21])
        wl = H.with_margin(oracle_mod, wl)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        orc.set_particles(H.oracle_particles(oracle_mod, wl))
        _sync_populations(gpu, orc, rng)
        gpu.step(1)
        orc.step(1)
        assert gpu.counters()["nrefill"] == orc.counters()["nrefill"]
        refilled += orc.counters()["nrefill"]
        own = orc.owner()
        assert np.array_equal(gpu.flags().cpu().numpy() - 1, own)
        err = np.abs(gpu.populations().cpu().numpy() - orc.populations())[:, own < 0].max()
        assert err <= POP_TOL[storage]
    assert refilled > 20


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_static_geometry_skips_flag_pass(pkg, oracle_mod, W, storage):
    """All particles fixed: from the fourth step on the flag pass is left out
    (the flags cannot change) and, below FP64, the fixed-geometry sweep runs
    (links and their geometry recorded once); five steps still agree with the
    oracle, which classifies every step.  Setting the particles again (moved, still
    fixed) brings the pass back: the moved geometry's flags, refilled nodes
    and populations agree after two more steps.  Tolerances: those of one
    step, times the number of steps."""
    wl = H.with_margin(oracle_mod, wl_touching(W))
    gpu = H.make_gpu(pkg, wl, storage=storage)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    _sync_populations(gpu, orc, np.random.default_rng(4))
    k_full = gpu.kernels_per_step()
    for _ in range(5):
        gpu.step(1)
        orc.step(1)
    # FP64: the brick sweeps without the flag pass; below FP64 the
    # fixed-geometry sweep (its link and plain kernels)
    assert gpu.kernels_per_step() == (k_full - 1 if storage == "f64" else 2)
    own = orc.owner()
    assert np.array_equal(gpu.flags().cpu().numpy() - 1, own)
    err = np.abs(gpu.populations().cpu().numpy() - orc.populations())[:, own < 0].max()
    assert err <= 5 * POP_TOL[storage], err
    Fg, _ = gpu.forces()
    Fo, _ = orc.forces()
    nl = orc.counters()["nlinks"]
    ftol = (1e-11 * nl * 0.2 if storage == "f64" else POP_TOL[storage] * nl + 1e-5 * np.abs(Fo).max())
    assert np.abs(Fg - Fo).max() <= 5 * ftol, (Fg, Fo)
    # move the first particle (still fixed): the flags must follow
    wl["particles"][0]["x"] = wl["particles"][0]["x"] + np.array([0.6, -0.4, 0.3])
    wl = H.with_margin(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    assert gpu.kernels_per_step() == k_full
    refilled = 0
    for _ in range(2):
        gpu.step(1)
        orc.step(1)
        assert gpu.counters()["nrefill"] == orc.counters()["nrefill"]
        refilled += orc.counters()["nrefill"]
    assert refilled > 5
    own = orc.owner()
    assert np.array_equal(gpu.flags().cpu().numpy() - 1, own)
    err = np.abs(gpu.populations().cpu().numpy() - orc.populations())[:, own < 0].max()
    assert err <= 7 * POP_TOL[storage], err


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("case", ["touching", "multi", "wrap"])
def test_fixed_geometry_sweep_same_bits(pkg, W, case, storage):
    """The fixed-geometry sweep (every particle fixed, from the fourth step)
    and the brick sweeps (the same particles not fixed, with no DEM
    sub-steps, so they do not move either) run the same arithmetic: after
    ten steps populations and force/torque totals are bit-identical."""
    wl = _case(W, case)
    runs = []
    for fixed in (1, 0):
        for p in wl["particles"]:
            p["fixed"] = fixed
        gpu = H.make_gpu(pkg, wl, storage=storage, n_sub=0)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        gpu.step(10)
        runs.append((gpu.populations().cpu().numpy(), *gpu.forces(), gpu.kernels_per_step()))
    (f1, F1, T1, k1), (f0, F0, T0, k0) = runs
    assert k1 == 2 and k0 == 5, (k1, k0)  # brick sweeps: binning, flags, plain, near, near-set plain bricks
    assert np.array_equal(f1, f0)
    assert np.array_equal(F1, F0) and np.array_equal(T1, T0)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("case", ["periodic_empty", "walls_guo_ragged"])
def test_empty_lattice_fixed_geometry_steps(pkg, oracle_mod, W, case, storage):
    """No particles (a fixed geometry with no links): from the fourth step
    the fixed-geometry sweep runs every node through its plain kernel; six
    steps agree with the oracle (one-step tolerance times the steps)."""
    wl = _case(W, case)
    gpu = H.make_gpu(pkg, wl, storage=storage)
    orc = H.make_oracle(oracle_mod, wl)
    _sync_populations(gpu, orc, np.random.default_rng(6))
    gpu.step(6)
    orc.step(6)
    assert gpu.kernels_per_step() == 2
    err = np.abs(gpu.populations().cpu().numpy() - orc.populations()).max()
    assert err <= 6 * POP_TOL[storage], err


def test_settling_sphere_trajectory_fp64(pkg, oracle_mod, W):
    """Workload 1 (sphere of §3.1 geometry, FP64), 12 steps with 100 DEM
    sub-steps each: particle state, force and populations agree."""
    wl = W.settling_sphere()
    wl["gravity"] = (0.0, 0.0, -2e-3)   # faster, so the 12 steps move it
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    for _ in range(12):
        gpu.step(1)
        orc.step(1)
    sg, so = gpu.particles()[0], orc.get_particles()[0]
    assert abs(sg["mass"] - so["mass"]) < 1e-9 * so["mass"]
    assert np.abs(sg["x"] - so["x"]).max() < 1e-10
    assert np.abs(sg["v"] - so["v"]).max() < 1e-11
    assert np.abs(sg["x"] - np.array([15.5, 15.5, 34.0])).max() > 1e-3
    Fg, Tg = gpu.forces()
    Fo, To = orc.forces()
    assert np.abs(Fg - Fo).max() < 1e-9 * max(1.0, np.abs(Fo).max())
    own = orc.owner()
    assert np.array_equal(gpu.flags().cpu().numpy() - 1, own)
    assert np.abs(gpu.populations().cpu().numpy() - orc.populations())[:, own < 0].max() < 1e-12


def test_settling_metaball_trajectory_fp32(pkg, oracle_mod, W):
    """A reduced box of workload 2 (FP32), 20 steps with DEM: the force
    history stays within FP32 accumulation error of the oracle's."""
    wl = W.settling_metaball(nx=48, ny=48, nz=64, steps=20)
    wl["particles"][0]["x"] = np.array([23.7, 24.2, 40.3])
    wl["gravity"] = (0.0, 0.0, -5e-3)
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    for _ in range(20):
        gpu.step(1)
        orc.step(1)
        Fg, _ = gpu.forces()
        Fo, _ = orc.forces()
        assert np.abs(Fg - Fo).max() <= 1e-3 * np.abs(Fo).max() + 1e-4
    sg, so = gpu.particles()[0], orc.get_particles()[0]
    assert np.abs(sg["x"] - so["x"]).max() < 1e-4
    assert np.abs(sg["v"] - so["v"]).max() < 1e-5


@pytest.mark.parametrize("storage,n_sub,w0,dem_mode", [("f64", 100, 0.02, 0), ("f32", 100, 0.02, 0),
                                                         ("f32", 1, 0.4, 0), ("bf16", 100, 0.02, 0),
                                                         ("f32", 100, 0.02, 1), ("f32", 1, 0.4, 1),
                                                         ("bf16", 100, 0.02, 1)])
def test_free_rotation(pkg, oracle_mod, W, storage, n_sub, w0, dem_mode):
    """Torque-free rotation of an asymmetric body (Euler's equations, §2.3.4):
    a metaball whose surface encloses the whole periodic box has no fluid
    links, so the hydrodynamic load is exactly zero and only the rotation
    sub-steps act.  With the FP64 rigid-body integrator (dem_mode 0, any
    storage) the attitude and w agree with the oracle to rounding (1e-12).
    The compensated-FP32 integrator (dem_mode 1, below FP64) computes each of
    the n_s increments (size ~|w| h / 2) with a relative error ~6e-8, so
    after S steps the attitude is off by at most ~S n_s * 6e-8 * |w| h / 2 =
    3e-8 S |w| (n_s h = 1), and w, whose increments are of order |w|^2 h
    here, by that times |w|; the test allows four times these (plus 3e-7 |w|
    for the FP32 rotation of the reported w to the world frame).  n_s = 1
    with |w| = 0.4 takes the large-angle branch of the exponential map."""
    inertia = np.array([[40.0, 3.0, -2.0], [3.0, 25.0, 1.5], [-2.0, 1.5, 12.0]])
    wl = W.empty_box(16, storage, (1, 1, 1))
    wl.update(n_sub=n_sub, gravity=(0.0, 0.0, -1e-4))
    wl["particles"] = [W._particle([[0.0, 0.0, 0.0], [1.0, 0.5, 0.0]], [4e4, 1e4], (8.3, 7.9, 8.1),
                                   q=(0.9, 0.1, -0.3, 0.2), v=(0.01, 0.0, 0.0), w=(w0, -0.6 * w0, 0.3 * w0),
                                   density=2.0, mass=500.0, inertia=inertia)]
    gpu = H.make_gpu(pkg, wl, dem_mode=dem_mode)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    for _ in range(10):
        gpu.step(1)
        orc.step(1)
    assert np.all(gpu.flags().cpu().numpy() == 1)
    Fg, Tg = gpu.forces()
    assert not Fg.any() and not Tg.any()
    sg, so = gpu.particles()[0], orc.get_particles()[0]
    qg = sg["q"] * np.sign(np.dot(sg["q"], so["q"]))
    steps = 10
    fp64 = storage == "f64" or dem_mode == 0
    tol_q = 1e-12 if fp64 else 4 * 3e-8 * steps * w0
    # the compensated integrator rotates the reported world-frame w out of
    # the principal frame in FP32 (relative error ~1e-7)
    tol_w = 1e-12 * w0 if fp64 else tol_q * w0 + 3e-7 * w0
    assert np.abs(qg - so["q"]).max() < tol_q
    assert np.abs(sg["w"] - so["w"]).max() < tol_w
    # translation: the compensated integrator takes the acceleration
    # (1 - rho0/rho_s) g in FP32 (relative 6e-8, the same every step), so v
    # drifts by up to S |a| 6e-8 and x by S^2/2 of that per step; the test
    # allows twice these
    acc = 0.5 * 1e-4
    tol_v = 1e-13 if fp64 else 2 * steps * acc * 6e-8
    tol_x = 1e-12 if fp64 else 2 * 0.5 * steps * steps * acc * 6e-8
    assert np.abs(sg["x"] - so["x"]).max() < tol_x
    assert np.abs(sg["v"] - so["v"]).max() < tol_v
    # the body really tumbles: w is not conserved in the world frame
    assert np.abs(so["w"] - np.array([w0, -0.6 * w0, 0.3 * w0])).max() > 1e-3 * w0


def test_set_particles_new_inertia(pkg, oracle_mod, W):
    """lbm_set_particles keeps each slot's principal-axes decomposition while
    its inertia tensor stays the same; a new tensor in the same slot is
    decomposed again.  After a first set of particles and two steps, the slot
    gets another tensor (same shape and pose): the torque-free rotation that
    follows agrees with the oracle's for that tensor to rounding (FP64
    integrator), which a reused decomposition would not."""
    I1 = np.array([[40.0, 3.0, -2.0], [3.0, 25.0, 1.5], [-2.0, 1.5, 12.0]])
    I2 = np.array([[18.0, -4.0, 1.0], [-4.0, 33.0, 2.5], [1.0, 2.5, 27.0]])
    wl = W.empty_box(16, "f32", (1, 1, 1))
    wl.update(n_sub=100, gravity=(0.0, 0.0, -1e-4))

    def parts(inertia):
        return [W._particle([[0.0, 0.0, 0.0], [1.0, 0.5, 0.0]], [4e4, 1e4], (8.3, 7.9, 8.1),
                            q=(0.9, 0.1, -0.3, 0.2), v=(0.01, 0.0, 0.0), w=(0.02, -0.012, 0.006),
                            density=2.0, mass=500.0, inertia=inertia)]
    wl["particles"] = parts(I1)
    gpu = H.make_gpu(pkg, wl, dem_mode=0)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    gpu.step(2)
    wl["particles"] = parts(I2)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc = H.make_oracle(oracle_mod, wl)
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    for _ in range(5):
        gpu.step(1)
        orc.step(1)
    sg, so = gpu.particles()[0], orc.get_particles()[0]
    qg = sg["q"] * np.sign(np.dot(sg["q"], so["q"]))
    assert np.abs(qg - so["q"]).max() < 1e-12
    assert np.abs(sg["w"] - so["w"]).max() < 1e-12 * 0.02


def test_full_size_settling_metaball_one_step(pkg, oracle_mod, W):
    """Workload 2 at its full 128x128x256 size in the benchmark's launch
    configuration: one step from a perturbed state, every fluid node and the
    force compared."""
    wl = W.settling_metaball()
    p = wl["particles"][0]
    p["v"] = np.array([0.004, -0.003, -0.02])
    p["w"] = np.array([0.001, 0.002, -0.001])
    wl = H.with_margin(oracle_mod, wl)
    _compare_step(pkg, oracle_mod, wl, "f32", amp=5e-3)


def test_deterministic(pkg, oracle_mod, W):
    wl = H.with_margin(oracle_mod, wl_multi(W))
    outs = []
    for _ in range(2):
        gpu = H.make_gpu(pkg, wl, n_sub=0)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        gpu.step(3)
        F, T = gpu.forces()
        outs.append((F, T, gpu.populations().cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_plain_speculation_same_bits(pkg, oracle_mod, W, storage):
    """Issuing the plain sweep's pulls before its near-set entry is read
    (mode 1) or after (mode 0) changes only the order of loads: three steps
    of a moving multi-particle case (walls and wraps, near bricks both ways)
    give bit-identical populations and forces, and the same as the default."""
    wl = H.with_margin(oracle_mod, wl_multi(W))
    outs = []
    for mode in (1, 0, -1):
        gpu = H.make_gpu(pkg, wl, storage=storage)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        gpu.set_plain_speculation(mode)
        gpu.step(3)
        F, T = gpu.forces()
        outs.append((F, T, gpu.populations().cpu().numpy()))
    for F, T, f in outs[1:]:
        assert np.array_equal(F, outs[0][0]) and np.array_equal(T, outs[0][1])
        assert np.array_equal(f, outs[0][2])
    with pytest.raises(pkg.LbmError):
        gpu.set_plain_speculation(2)


def test_profile_mask_records_chosen_kernels(pkg, oracle_mod, W):
    """Profiling every kernel records the binning, flags, plain and near
    sweeps of each step; with only the plain sweep named, four further steps
    record it four times and nothing else; sampling every third launch
    records three of seven."""
    wl = H.with_margin(oracle_mod, wl_multi(W))
    gpu = H.make_gpu(pkg, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    gpu.profile(True)
    gpu.step(2)
    rec = gpu.profile_read()
    gpu.profile(False)
    assert all(rec[k][1] == 2 for k in ("k_bin", "k_flags", "k_sweep_plain", "k_sweep_near")), rec
    gpu.profile(True, kernels=["k_sweep_plain"])
    gpu.step(4)
    rec = gpu.profile_read()
    gpu.profile(False)
    assert rec["k_sweep_plain"][1] == 4
    assert all(n == 0 for k, (_, n) in rec.items() if k != "k_sweep_plain"), rec
    # a sample: launches 0, 3 and 6 of seven
    gpu.profile(True, kernels=["k_sweep_plain"], every=3)
    gpu.step(7)
    rec = gpu.profile_read()
    gpu.profile(False)
    assert rec["k_sweep_plain"][1] == 3 and rec["k_sweep_plain"][0] > 0, rec


def test_back_to_back_steps_same_bits(pkg, oracle_mod, W):
    """Steps issued back to back in one call (the plain sweep and the near
    set's link-free bricks of step t then run beside the DEM, binning and flag
    pass of t+1) give the same bits as the same steps issued one at a time
    with the device idle in between: twelve moving metaballs in a 64x64x96
    box, DEM on, twelve steps; flags, populations, forces and torques equal."""
    wl = W.multi_particle(12, n=64, nz=96, storage="f32", steps=12, seed_offset=11)
    rng = np.random.default_rng(12)
    for p in wl["particles"]:
        p["v"] = rng.uniform(-0.02, 0.02, 3)
        p["w"] = rng.uniform(-0.002, 0.002, 3)
    wl = H.with_margin(oracle_mod, wl)
    runs = []
    for together in (True, False):
        gpu = H.make_gpu(pkg, wl)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        if together:
            gpu.step(12)
        else:
            for _ in range(12):
                gpu.step(1)
                torch.cuda.synchronize()
        runs.append((gpu.flags().cpu().numpy(), gpu.populations().cpu().numpy(), *gpu.forces()))
    (la, fa, Fa, Ta), (lb, fb, Fb, Tb) = runs
    assert np.array_equal(la, lb)
    assert np.array_equal(fa, fb)
    assert np.array_equal(Fa, Fb) and np.array_equal(Ta, Tb)


def test_mass_conserved_closed_box_fp64(pkg, W):
    wl = wl_walls_guo_ragged(W)
    wl["force"] = (0.0, 0.0, 0.0)
    gpu = H.make_gpu(pkg, wl, storage="f64")
    rng = np.random.default_rng(0)
    f = rng.uniform(0.99, 1.01, (19,) + gpu.shape) / 19
    gpu.set_populations(torch.from_numpy(f).cuda())
    m0 = gpu.populations().sum().item()
    gpu.step(50)
    assert abs(gpu.populations().sum().item() - m0) < 1e-13 * m0


def test_brick_overflow_reported(pkg, W):
    """More particles than one brick's list holds: reported, not silent."""
    wl = W.empty_box(8, "f32", (1, 1, 1))
    wl.update(nx=32, ny=16, nz=16)
    wl["particles"] = [W._particle([[0, 0, 0]], [1.0], (1.0 + 1.7 * k, 2.0, 1.0), fixed=1) for k in range(17)]
    H.fixed_mass(wl)
    gpu = H.make_gpu(pkg, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    gpu.step(1)
    with pytest.raises(pkg.LbmError) as e:
        gpu.forces()
    assert e.value.code == -3


def test_divergence_reported(pkg, W):
    gpu = H.make_gpu(pkg, wl_periodic_empty(W))
    f = gpu.populations()
    f[3, 2, 3, 4] = float("nan")
    gpu.set_populations(f)
    gpu.step(1)
    with pytest.raises(pkg.LbmError) as e:
        gpu.check()
    assert e.value.code == -4
