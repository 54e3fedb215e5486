"""CPU checks of the seeded input generators (host code only)."""
import numpy as np

from paper_2206_11634_gb300 import workloads as W


def _check_placement(wl):
    per = wl["periodic"]
    L = np.array([wl["nx"], wl["ny"], wl["nz"]], dtype=float)
    cs = [p["x"] for p in wl["particles"]]
    bs = [W.bounding_radius(p["cp"], p["K"], p["Rs"]) for p in wl["particles"]]
    for i in range(len(cs)):
        for a in range(3):
            if not per[a]:
                assert bs[i] < cs[i][a] < L[a] - 1 - bs[i]
        for j in range(i):
            d = cs[i] - cs[j]
            for a in range(3):
                if per[a]:
                    d[a] -= L[a] * np.round(d[a] / L[a])
            assert np.linalg.norm(d) >= bs[i] + bs[j] + 2.0 - 1e-12


def test_multi_particle_full_size_placement_and_seed():
    a = W.multi_particle()
    b = W.multi_particle()
    assert len(a["particles"]) == 200
    _check_placement(a)
    for p, q in zip(a["particles"], b["particles"]):
        assert np.array_equal(p["x"], q["x"]) and np.array_equal(p["K"], q["K"])
    ncp = [len(p["K"]) for p in a["particles"]]
    assert min(ncp) >= 2 and max(ncp) <= 8
    # sum K = R^2 with the nominal radius in [5, 8]
    R = [np.sqrt(p["K"].sum()) for p in a["particles"]]
    assert 5.0 <= min(R) and max(R) <= 8.0


def test_small_multi_particle_cases_place():
    for count, n, nz in [(10, 64, 64), (8, 64, 48)]:
        _check_placement(W.multi_particle(count, n=n, nz=nz, seed_offset=7))


def test_settling_metaball_shape():
    wl = W.settling_metaball()
    p = wl["particles"][0]
    assert p["cp"].shape == (4, 3) and np.abs(p["cp"]).max() <= 4.0
    assert 9.0 <= p["K"].min() and p["K"].max() <= 25.0
    assert (wl["nx"], wl["ny"], wl["nz"]) == (128, 128, 256)
    _check_placement(wl)


def test_settling_sphere():
    wl = W.settling_sphere()
    p = wl["particles"][0]
    assert p["K"][0] == 36.0 and (wl["nx"], wl["ny"], wl["nz"]) == (32, 32, 48) and wl["storage"] == "f64"
