"""GPU parity of the DEM with contacts (§2.1, §2.3.4): metaball-metaball and
metaball-wall contacts, their onset and release, tangential springs, and the
closing half-kick, against the FP64 oracle over several LBM steps of 100
sub-steps.

Modes (lbm_config.dem_mode): FP64 lattice (everything FP64); FP32 lattice
with the default FP64 rigid-body integrator and FP32 contact geometry (0),
with the compensated-FP32 integrator (1), and with FP64 contact geometry as
well (2).  The pile of 34 particles takes the 512-thread paths of the
FP32-geometry kernels (more than 16 or 32 particles).

Tolerances:
- FP64: contact forces within 1e-8 of their scale, positions 1e-9,
  velocities 1e-10 (both sides converge the contact Newton iterations to
  1e-12 and integrate the same sub-steps; only rounding order differs).
- FP32 lattice: the hydrodynamic load differs from the oracle's by ~1e-5
  relative, the FP32 contact geometry puts ~1e-6 lu on an overlap of
  ~0.05 lu (2e-5 relative), and four steps of contact dynamics
  (k_n/m t^2 ~ 8) amplify both to ~1e-4; the test allows 2e-3 of the force
  scale, 2e-5 lu in position and 1e-5 in velocity.
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


def wl_trio(W, storage):
    """A sphere resting on the bottom wall (overlap ~0.013 lu of the contact
    skin) and two touching two-control-point metaballs (overlap ~0.16 lu)."""
    wl = W.empty_box(8, storage, (1, 1, 0))
    wl.update(nx=48, ny=40, nz=36, tau=0.8, n_sub=100, gravity=(0.0, 0.0, -1e-3),
              kn=200.0, eta_n=5.0, kt=100.0, eta_t=2.0, mu_s=0.3, c_tol=1e-6)
    I = np.array([[7000.0, 300.0, -150.0], [300.0, 6500.0, 100.0], [-150.0, 100.0, 6000.0]])
    cpB = [[0.8, 0.0, 0.3], [-0.8, 0.1, -0.3]]
    wl["particles"] = [
        W._particle([[0, 0, 0]], [25.0], (10.3, 20.1, 4.93), density=1.3, Rs=0.5, mass=700.0, inertia=I,
                    v=(0.003, 0.0, -0.004), w=(0.0, 0.002, 0.0)),
        W._particle(cpB, [9.0, 7.0], (26.2, 18.7, 18.4), density=1.3, Rs=0.5, mass=600.0, inertia=I * 0.55,
                    q=(0.9, 0.2, -0.1, 0.3), v=(0.004, 0.0, 0.001), w=(0.001, 0.0, -0.002)),
        W._particle(cpB, [8.0, 8.0], (35.1, 19.0, 18.9), density=1.3, Rs=0.5, mass=600.0, inertia=I * 0.5,
                    q=(0.7, -0.3, 0.2, 0.5), v=(-0.004, 0.001, 0.0), w=(0.0, 0.001, 0.001)),
    ]
    return wl


def wl_pile(W, oracle_mod, storage, target=0.03, side=3):
    """A side x side layer of spheres on the floor (overlaps ~0.05 lu with
    the floor and each other) and (side-1)^2 two-control-point metaballs
    lowered onto it until their largest overlap reaches `target` (placed with
    the oracle's pair geometry): 13 particles for side 3, 41 for side 5."""
    rng = np.random.default_rng(42)
    wl = W.empty_box(8, storage, (1, 1, 0))
    r, pitch = 4.5, 9.83
    n = int(np.ceil(12.0 + (side - 1) * pitch))
    wl.update(nx=n, ny=n, nz=32, tau=0.8, n_sub=100, gravity=(0.0, 0.0, -1e-3),
              kn=200.0, eta_n=5.0, kt=100.0, eta_t=2.0, mu_s=0.3, c_tol=1e-6)
    parts = []
    for iy in range(side):
        for ix in range(side):
            x = (6.0 + ix * pitch + 0.01 * iy, 6.0 + iy * pitch, r - 0.5 + 0.39)
            parts.append(W._particle([[0, 0, 0]], [r * r], x, density=1.3, Rs=0.5))
    for iy in range(side - 1):
        for ix in range(side - 1):
            ax = rng.normal(size=3)
            ax /= np.linalg.norm(ax)
            x = (6.0 + (ix + 0.5) * pitch, 6.0 + (iy + 0.5) * pitch, 12.0)
            parts.append(W._particle([0.5 * ax, -0.5 * ax], [r * r / 2, r * r / 2 - 1.0], x, density=1.3, Rs=0.5,
                                     v=(0.0, 0.0, -0.002), w=(0.001 * ix, -0.001, 0.0)))
    for p in parts:
        m = 1.3 * 4.0 / 3.0 * np.pi * r ** 3
        p["mass"] = m
        p["inertia"] = np.diag([0.4 * m * r * r, 0.41 * m * r * r, 0.39 * m * r * r])
    wl["particles"] = parts
    orc = H.make_oracle(oracle_mod, wl)
    nb = side * side
    for k in range(nb, len(parts)):
        z = parts[0]["x"][2] + 2 * r + 1.5
        while True:
            parts[k]["x"][2] = z
            orc.set_particles(H.oracle_particles(oracle_mod, wl))
            hits = [orc.pair_geometry(i, k) for i in range(nb)]
            dmax = max([h[1] for h in hits if h[0]] or [-1.0])
            if dmax >= target:
                break
            z -= 0.01
    return wl


MODES = [("f64", 0), ("f32", 0), ("f32", 1), ("f32", 2)]


@pytest.mark.parametrize("storage,dem_mode", MODES)
@pytest.mark.parametrize("case", ["trio", "pile", "pile41"])
def test_contact_trajectory(pkg, oracle_mod, W, case, storage, dem_mode):
    if case == "trio":
        wl = wl_trio(W, storage)
    else:
        wl = wl_pile(W, oracle_mod, storage, side=5 if case == "pile41" else 3)
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl, storage=storage, dem_mode=dem_mode)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    f64 = storage == "f64"
    tolF, tolx, tolv = (1e-8, 1e-9, 1e-10) if f64 else (2e-3, 2e-5, 1e-5)
    active = 0
    for _ in range(4):
        gpu.step(1)
        orc.step(1)
        Fg, Tg = gpu.contact_forces()
        Fo, To = orc.contact_forces()
        scale = max(1.0, np.abs(Fo).max())
        active += int(np.count_nonzero(np.abs(Fo).sum(1)))
        assert np.abs(Fg - Fo).max() <= tolF * scale, (np.abs(Fg - Fo).max(), scale)
        # lever arms up to ~6 lu
        assert np.abs(Tg - To).max() <= 10 * tolF * scale, (np.abs(Tg - To).max(), scale)
        Hg, _ = gpu.forces()
        Ho, _ = orc.forces()
        assert np.abs(Hg - Ho).max() <= (1e-9 if f64 else 1e-3) * max(1.0, np.abs(Ho).max())
    assert active >= {"trio": 5, "pile": 20, "pile41": 80}[case]
    for sg, so in zip(gpu.particles(), orc.get_particles()):
        assert np.abs(sg["x"] - so["x"]).max() < tolx, (sg["x"], so["x"])
        assert np.abs(sg["v"] - so["v"]).max() < tolv, (sg["v"], so["v"])
        qg = sg["q"] * np.sign(np.dot(sg["q"], so["q"]))
        assert np.abs(qg - so["q"]).max() < 10 * tolx
        assert np.abs(sg["w"] - so["w"]).max() < 10 * tolv
    own = orc.owner()
    assert np.array_equal(gpu.flags().cpu().numpy() - 1, own)


def test_contact_free_fall_has_no_contact_load(pkg, oracle_mod, W):
    """A particle far from everything: contact forces are exactly zero on both
    sides, whichever DEM runs."""
    wl = wl_trio(W, "f32")
    wl["particles"] = wl["particles"][1:2]
    wl["particles"][0]["x"] = np.array([24.0, 20.0, 18.0])
    wl = H.with_margin(oracle_mod, wl)
    for dem_mode in (0, 1, 2):
        gpu = H.make_gpu(pkg, wl, dem_mode=dem_mode)
        gpu.set_particles(H.gpu_particles(pkg, wl))
        gpu.step(2)
        F, T = gpu.contact_forces()
        assert not F.any() and not T.any()
