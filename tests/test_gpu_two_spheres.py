"""§3.3's two-sphere comparison: without the missing-force-point treatment
(§2.3.5 item 2, Eqs. (31)-(32)) spheres close to a wall and to each other
spin up for no physical reason; with it they do not.  GPU (FP32 lattice,
default DEM) and the FP64 oracle side by side.

- At rest: two spheres of radius 6 resting on the floor (covering the first
  node layer) 0.25 nodes apart, fluid at rest, no gravity and no contact
  spring.  Physically nothing moves.  With the treatment the force and torque
  on each sphere are zero (the oracle's to rounding, the GPU's exactly in its
  offset form) and |w| stays below 1e-12 for 50 steps.  Without it the
  anisotropic force points give each sphere a spurious force and torque from
  the first step and the spin grows (|w| at step 50 more than 5 times that at
  step 2, above 1e-4); the GPU follows the oracle's spin to 1e-3 relative.
- Settling: the same pair under gravity with a contact spring, from just
  above the floor, 1000 steps: with the treatment the spin the settling
  causes dies away; without it it stays several times larger (by step 1000,
  on both sides, at least 3 times the treated mean |w| over the last 100
  steps), and the first 100 steps agree between GPU and oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

R = 6.0


@pytest.fixture(scope="module")
def pkg():
    from paper_2206_11634_gb300 import build as b
    b.build()
    import paper_2206_11634_gb300 as p
    return p


# sphere centres: resting pair (0.25 nodes apart, both covering the first
# node layer) and settling pair (0.65 apart, just above the contact skin)
AT_REST = ((13.3, 16.2, 5.63), (25.55, 15.7, 5.77))
SETTLING = ((13.3, 16.2, 5.93), (25.95, 15.7, 6.07))


def _pair(make, centres):
    m = 2.5 * 4.0 / 3.0 * np.pi * R ** 3
    I = np.eye(3) * 0.4 * m * R * R
    return [make([[0, 0, 0]], [R * R], c, density=2.5, mass=m, inertia=I, Rs=0.5) for c in centres]


def _both(pkg, oracle_mod, mf, n, **phys):
    kw = dict(periodic=(0, 0, 0), tau=0.8, missing_force=mf, c_tol=1e-6, **phys)
    gpu = pkg.Lattice(*n, lattice=19, storage="f32", max_particles=2, **kw)
    orc = oracle_mod.Oracle(*n, Q=19, **kw)
    return gpu, orc


def _spin(states):
    return max(float(np.linalg.norm(s["w"])) for s in states)


@pytest.mark.parametrize("mf", [1, 0])
def test_two_spheres_at_rest_spurious_spin(pkg, oracle_mod, mf):
    gpu, orc = _both(pkg, oracle_mod, mf, (40, 32, 28), n_sub=20, gravity=(0.0, 0.0, 0.0))
    gpu.set_particles(_pair(pkg.make_particle, AT_REST))
    orc.set_particles(_pair(oracle_mod.make_particle, AT_REST))
    assert orc.min_margin() > 1e-9
    wg, wo = [], []
    for _ in range(50):
        gpu.step(1)
        orc.step(1)
        wg.append(_spin(gpu.particles()))
        wo.append(_spin(orc.get_particles()))
    if mf:
        Fg, Tg = gpu.forces()
        assert not Fg.any() and not Tg.any()       # offset form: exactly zero
        assert max(wg) < 1e-12 and max(wo) < 1e-12, (max(wg), max(wo))
    else:
        assert wo[-1] > 5 * wo[1] and wo[-1] > 1e-4, wo
        assert wg[-1] > 5 * wg[1] and wg[-1] > 1e-4, wg
        assert np.allclose(wg, wo, rtol=1e-3, atol=1e-9), (wg[-1], wo[-1])


def test_two_spheres_settling_spin(pkg, oracle_mod):
    late = {}
    for mf in (1, 0):
        gpu, orc = _both(pkg, oracle_mod, mf, (40, 32, 40), n_sub=50, gravity=(0.0, 0.0, -2e-4), kn=50.0,
                         eta_n=2.0, kt=25.0, eta_t=1.0, mu_s=0.3)
        gpu.set_particles(_pair(pkg.make_particle, SETTLING))
        orc.set_particles(_pair(oracle_mod.make_particle, SETTLING))
        wg, wo = [], []
        for step in range(1000):
            gpu.step(1)
            orc.step(1)
            wg.append(_spin(gpu.particles()))
            wo.append(_spin(orc.get_particles()))
            if step == 99:
                for sg, so in zip(gpu.particles(), orc.get_particles()):
                    assert np.abs(sg["x"] - so["x"]).max() < 2e-4, (sg["x"], so["x"])
                    assert np.abs(sg["w"] - so["w"]).max() < 2e-5, (sg["w"], so["w"])
        late[mf] = (np.mean(wg[-100:]), np.mean(wo[-100:]))
    assert late[0][0] > 3 * late[1][0], late
    assert late[0][1] > 3 * late[1][1], late
