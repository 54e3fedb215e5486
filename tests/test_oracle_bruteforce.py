"""The oracle's whole lattice step against a brute-force transcription.

tests/_bruteforce.py restates one step of the method from the paper (§2.2,
§2.3: classification by Eq. (26), refilling Eq. (30), pull streaming with
halfway walls, VIBB Eqs. (19)-(25) with the q of Eq. (27) and the halfway
fallback of §2.3.5 item 1, BGK Eqs. (14)-(16) with Guo forcing, the momentum
exchange Eqs. (28)-(29) and the missing force points Eqs. (31)-(32)) in plain
Python loops over every node, link and particle, sharing nothing with
oracle/lbm_oracle.c.  On grids of at most 8^3 nodes the two must agree to
1e-14 in every fluid population, exactly in the node owners and the link and
refill counts, and to 1e-14 of the force scale in the force and torque
totals, over several steps in which the particles move (so that nodes are
uncovered and refilled):

- a moving three-control-point metaball between two walls, periodic in y and
  z, with a body force;
- two overlapping metaballs touching a wall (nodes covered twice, links
  whose far node is beyond the wall or inside the other particle, VIBB
  falling back to halfway bounce-back);
- a metaball straddling the corner of a fully periodic box (every link and
  distance by minimum image).
"""
import numpy as np
import pytest

from tests import _bruteforce as bf


def _perm(o):
    """perm[k]: the transcription's index of the oracle's direction k."""
    return np.array([int(np.flatnonzero((bf.E == o.e[k]).all(axis=1))[0]) for k in range(o.Q)])


def _oracle_particle(oracle_mod, p):
    return oracle_mod.make_particle(p["cp"], p["K"], p["x"], q=p["q"], v=p["v"], w=p["w"], mass=10.0,
                                    inertia=np.eye(3) * 40.0, fixed=1)


def _unit(q):
    q = np.asarray(q, dtype=np.float64)
    return q / np.sqrt(q @ q)


CASES = {
    "moving_metaball": dict(
        shape=(8, 7, 6), periodic=(0, 1, 1), tau=0.7, force=(2e-4, 0.0, -1e-4),
        particles=[dict(cp=[[1.1, 0.2, -0.3], [-0.9, 0.5, 0.4], [0.1, -0.8, 0.2]], K=[1.2, 0.9, 1.0],
                        x=[3.4, 3.1, 2.7], q=_unit([0.9, 0.2, -0.3, 0.1]), v=[0.05, -0.03, 0.02],
                        w=[0.01, 0.02, -0.015])],
        moves=[[0.45, -0.35, 0.3], [0.4, 0.3, -0.35]], exercises=("nhalfway",)),
    "touching_pair_at_wall": dict(
        shape=(8, 8, 8), periodic=(0, 0, 0), tau=0.8, force=(0.0, 0.0, 0.0),
        particles=[dict(cp=[[0.6, 0.0, 0.0], [-0.6, 0.1, 0.0]], K=[1.6, 1.4], x=[2.2, 3.6, 1.2],
                        q=_unit([0.95, 0.0, 0.2, 0.1]), v=[0.02, 0.01, -0.03], w=[0.0, 0.02, 0.01]),
                   dict(cp=[[0.0, 0.7, 0.2], [0.1, -0.6, -0.2]], K=[1.5, 1.3], x=[4.9, 3.9, 1.6],
                        q=_unit([0.8, 0.3, 0.0, -0.2]), v=[-0.03, 0.0, 0.02], w=[0.015, -0.01, 0.0])],
        moves=[[0.0, 0.5, -0.2], [0.3, -0.4, 0.1]], exercises=("nhalfway", "nmissing", "ndouble")),
    "periodic_corner": dict(
        shape=(7, 8, 6), periodic=(1, 1, 1), tau=0.9, force=(-1e-4, 1.5e-4, 5e-5),
        particles=[dict(cp=[[0.8, -0.4, 0.3], [-0.7, 0.6, -0.2], [0.0, 0.1, -0.9]], K=[1.0, 1.1, 0.8],
                        x=[0.3, 7.6, 5.7], q=_unit([0.7, -0.4, 0.5, 0.3]), v=[0.04, 0.03, -0.02],
                        w=[-0.02, 0.01, 0.03])],
        moves=[[-0.5, 0.4, 0.45], [-0.45, 0.35, 0.4]], exercises=()),
}


def _margin_ok(oracle_mod, case, parts, o):
    o.set_particles([_oracle_particle(oracle_mod, p) for p in parts])
    return o.min_margin() > 1e-9


@pytest.mark.parametrize("name", list(CASES))
def test_step_matches_bruteforce(oracle_mod, name):
    case = CASES[name]
    nx, ny, nz = case["shape"]
    o = oracle_mod.Oracle(nx, ny, nz, Q=19, periodic=case["periodic"], tau=case["tau"], force=case["force"])
    ref = bf.Step(case["shape"], case["periodic"], case["tau"], force=case["force"])
    perm = _perm(o)
    rng = np.random.default_rng(2206 + len(name))
    parts = [dict(p) for p in case["particles"]]
    f0 = rng.uniform(0.99, 1.01, (19, nz, ny, nx)) * o.w[:, None, None, None]
    f0[1] *= 1.01   # a little flow along +x
    o.set_populations(f0)
    ref.f[perm] = f0
    moves = [np.zeros(3)] + [np.asarray(m) for m in case["moves"]]
    seen = dict(nlinks=0, nrefill=0, nhalfway=0, nmissing=0, ndouble=0)
    for k, mv in enumerate(moves):
        for p in parts:
            p["x"] = np.asarray(p["x"], dtype=np.float64) + mv
        # keep every node at least 1e-9 (relative) away from a surface
        for _ in range(20):
            if _margin_ok(oracle_mod, case, parts, o):
                break
            for p in parts:
                p["x"] = p["x"] + rng.uniform(-1e-4, 1e-4, 3)
        else:
            raise RuntimeError("no margin")
        ref.set_particles(parts)
        o.step(1)
        ref.step()
        own = o.owner()
        assert np.array_equal(own, ref.own), f"{name} step {k}: node owners differ"
        fluid = own < 0
        fo = o.populations()[:, fluid]
        fb = ref.f[perm][:, fluid]
        assert np.abs(fo - fb).max() <= 1e-14, f"{name} step {k}: populations differ by {np.abs(fo - fb).max():.2e}"
        c = o.counters()
        assert c["nlinks"] == ref.nlinks and c["nrefill"] == ref.nrefill
        Fo, To = o.forces()
        scale = max(1.0, np.abs(ref.Fh).max(), np.abs(ref.Th).max())
        assert np.abs(Fo - ref.Fh).max() <= 1e-14 * scale
        assert np.abs(To - ref.Th).max() <= 1e-14 * scale
        for key in seen:
            seen[key] += getattr(ref, key)
    # the cases exercise what they are meant to
    assert seen["nlinks"] > 50 and seen["nrefill"] > 0
    for key in case["exercises"]:
        assert seen[key] > 0, (name, key, seen)
