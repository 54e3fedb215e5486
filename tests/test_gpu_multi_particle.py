"""GPU parity of the 200-metaball workload at its full 256^3 size (§4's
multi-particle run, scaled), in the benchmark's launch configuration.

- One step from a perturbed state (random populations w_i(1 + U(+-1 %)),
  every particle moving and turning): flags bit-exact, every fluid
  population within the FP32 one-step tolerance (2e-6), and the force and
  torque of all 200 particles within 2e-6 per link plus 1e-5 relative.
- A 20-step window with the DEM on (100 sub-steps, default FP64 rigid-body
  integrator with FP32 contact geometry) in which particles launched towards
  each other come into contact, both sides from the same start: per step the
  hydrodynamic force of every particle within 1e-3 of the largest plus 1e-3
  relative; after 20 steps positions within 2e-4 lu and velocities within
  5e-5 (FP32 force sums and FP32 contact geometry, amplified by the contact
  dynamics); flag differences caused by that divergence are counted and must
  stay below 1e-6 of the nodes (reported, not failed, when positions differ
  by rounding at a surface).
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


def _launch(wl, seed, vmax, wmax):
    rng = np.random.default_rng(seed)
    for p in wl["particles"]:
        p["v"] = rng.uniform(-vmax, vmax, 3)
        p["w"] = rng.uniform(-wmax, wmax, 3)
    return wl


def _approaching_pairs(oracle_mod, wl, npairs=3, gap=0.3, speed=0.03):
    """Move a few neighbouring particles (one of each pair, along the line of
    centres) until their skins are about `gap` apart, checked with the
    oracle's pair geometry, and set them approaching each other at `speed`:
    they touch within the window.  Only pairs of similar size (equivalent
    radii within 10 %: Eq. (5)'s constraint c_tol < M < 1 finds the contact of
    two metaballs of quite different sizes inside the larger one and rejects
    it, on both sides alike) whose moved particle stays clear of every other
    one are used."""
    parts = wl["particles"]
    # geometry only: a small walled lattice (no periodic images) will do; the
    # pairs are chosen by plain distance, so none straddles a periodic face
    orc = H.make_oracle(oracle_mod, dict(wl, nx=8, ny=8, nz=8, periodic=(0, 0, 0)))
    b = [_bound(p) for p in parts]
    used, done = set(), 0
    order = sorted(((np.linalg.norm(parts[i]["x"] - parts[j]["x"]) - b[i] - b[j], i, j)
                    for i in range(len(parts)) for j in range(i + 1, len(parts))))
    for _, i, j in order:
        if done == npairs:
            break
        if i in used or j in used:
            continue
        ri, rj = np.sqrt(np.sum(parts[i]["K"])), np.sqrt(np.sum(parts[j]["K"]))
        if abs(ri - rj) > 0.1 * max(ri, rj):
            continue
        u = parts[i]["x"] - parts[j]["x"]
        u /= np.linalg.norm(u)
        x0 = parts[j]["x"].copy()
        pi = dict(parts[i], mass=1.0, inertia=np.eye(3))
        for step in np.arange(0.0, 10.0, 0.05):
            pj = dict(parts[j], x=x0 + step * u, mass=1.0, inertia=np.eye(3))
            orc.set_particles(H.oracle_particles(oracle_mod, dict(particles=[pi, pj])))
            if orc.pair_geometry(0, 1)[0]:
                break
        else:
            parts[j]["x"] = x0
            continue
        parts[j]["x"] = x0 + max(0.0, step - gap) * u
        clear = all(np.linalg.norm(parts[j]["x"] - parts[k]["x"]) > b[j] + b[k] + 0.5
                    for k in range(len(parts)) if k not in (i, j))
        if not clear:
            parts[j]["x"] = x0
            continue
        parts[i]["v"] = -speed * u
        parts[j]["v"] = speed * u
        used.update((i, j))
        done += 1
    assert done == npairs
    return wl


def _bound(p):
    """Bounding radius about the centre: farthest control point + sqrt(sum K) + R_s."""
    return float(np.linalg.norm(np.asarray(p["cp"]), axis=1).max() + np.sqrt(np.sum(p["K"])) + p["Rs"])


def test_full_size_multi_particle_one_step(pkg, oracle_mod, W):
    wl = _launch(W.multi_particle(), 1, 0.02, 0.002)
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    rng = np.random.default_rng(3)
    f = rng.uniform(0.99, 1.01, (19,) + gpu.shape) * orc.w[:, None, None, None]
    gpu.set_populations(torch.from_numpy(f).cuda())
    del f
    orc.set_populations(gpu.populations().cpu().numpy())
    gpu.step(1)
    orc.step(1)
    own = orc.owner()
    assert np.array_equal(gpu.flags().cpu().numpy() - 1, own)
    fluid = own < 0
    err = 0.0
    fg = gpu.populations().cpu().numpy()
    fo = orc.populations()
    for i in range(19):  # per direction, to keep the temporaries small
        err = max(err, float(np.abs(fg[i][fluid] - fo[i][fluid]).max()))
    del fg, fo
    assert err <= 2e-6, err
    nl = orc.counters()["nlinks"]
    assert gpu.counters()["nlinks"] == nl and nl > 100000
    Fg, Tg = gpu.forces()
    Fo, To = orc.forces()
    # per particle: its own links (about nl / 200) at 2e-6 each, plus 1e-5 relative
    ftol = 2e-6 * nl / len(wl["particles"]) * 3 + 1e-5 * np.abs(Fo).max()
    assert np.abs(Fg - Fo).max() <= ftol, (np.abs(Fg - Fo).max(), ftol)
    assert np.abs(Tg - To).max() <= 20 * ftol


def test_multi_particle_window_with_contacts(pkg, oracle_mod, W):
    wl = _launch(W.multi_particle(), 2, 0.01, 0.002)
    wl = _approaching_pairs(oracle_mod, wl)
    wl = H.with_margin(oracle_mod, wl)
    gpu = H.make_gpu(pkg, wl)
    orc = H.make_oracle(oracle_mod, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    contacts = 0
    for _ in range(20):
        gpu.step(1)
        orc.step(1)
        Fg, _ = gpu.forces()
        Fo, _ = orc.forces()
        scale = np.abs(Fo).max()
        assert np.abs(Fg - Fo).max() <= 1e-3 * scale + 1e-3 * np.abs(Fo).max(), (np.abs(Fg - Fo).max(), scale)
        Co, _ = orc.contact_forces()
        contacts += int(np.count_nonzero(np.abs(Co).sum(1)))
    assert contacts > 0, "no contact in the window"
    for sg, so in zip(gpu.particles(), orc.get_particles()):
        assert np.abs(sg["x"] - so["x"]).max() < 2e-4, (sg["x"], so["x"])
        assert np.abs(sg["v"] - so["v"]).max() < 5e-5, (sg["v"], so["v"])
    flips = int(np.count_nonzero(gpu.flags().cpu().numpy() - 1 != orc.owner()))
    assert flips <= 1e-6 * wl["nx"] * wl["ny"] * wl["nz"], flips
    gpu.check()
