"""Batched lattices (lbm_batch_*): independent drag cases of different box
sizes stepped together, one launch per phase, the steps of a call as a
captured CUDA graph.

The batched kernels run the single-lattice bodies on each case's parameters,
so every case must agree bit for bit with the same case stepped alone
through lbm_step() (which the parity suite checks against the oracle), for
any launch schedule and any split of the steps into calls (graph replays).
One case is also compared with the FP64 oracle directly.
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


def cases(storage="f32", n=5):
    from paper_2206_11634_gb300 import workloads as W
    return W.batched_drag(n, storage, lo=24, hi=48, seed_offset=9)


def cfg_kw(wl):
    kw = {k: wl[k] for k in H.PHYS_KEYS}
    kw.update(nx=wl["nx"], ny=wl["ny"], nz=wl["nz"], periodic=tuple(wl["periodic"]), storage=wl["storage"],
              max_particles=1)
    return kw


def make_batch(pkg, wls):
    b = pkg.Batch([cfg_kw(wl) for wl in wls])
    for c, wl in enumerate(wls):
        b.set_particles(c, H.gpu_particles(pkg, wl))
    return b


def state(obj, c=None):
    if c is None:
        F, T = obj.forces()
        return obj.populations().cpu().numpy(), F, T
    F, T = obj.forces(c)
    return obj.populations(c).cpu().numpy(), F, T


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_matches_single_lattices(pkg, storage):
    wls = cases(storage)
    b = make_batch(pkg, wls)
    b.step(7)
    for c, wl in enumerate(wls):
        g = H.make_gpu(pkg, wl)
        g.set_particles(H.gpu_particles(pkg, wl))
        g.step(7)
        fb, Fb, Tb = state(b, c)
        fs, Fs, Ts = state(g)
        assert np.array_equal(fb, fs), f"case {c}: populations differ"
        assert np.array_equal(Fb, Fs) and np.array_equal(Tb, Ts), f"case {c}: forces differ"
        assert np.abs(Fs).max() > 0
    # all cases at once: the per-case rows, in case order
    Fa, Ta = b.all_forces()
    per = [b.forces(c) for c in range(len(wls))]
    assert np.array_equal(Fa, np.concatenate([F for F, _ in per]))
    assert np.array_equal(Ta, np.concatenate([T for _, T in per]))


def test_batch_graph_replay_and_schedule(pkg):
    wls = cases()
    a = make_batch(pkg, wls)
    for _ in range(3):
        a.step(3)  # captured once, replayed twice
    b = make_batch(pkg, wls)
    b.set_schedule(1, 1)
    b.step(9)
    c = make_batch(pkg, wls)
    c.set_schedule(8, 8)
    for _ in range(9):
        c.step(1)
    assert a.steps == b.steps == c.steps == 9
    for k in range(len(wls)):
        sa, sb, sc = state(a, k), state(b, k), state(c, k)
        for x, y, z in zip(sa, sb, sc):
            assert np.array_equal(x, y) and np.array_equal(x, z)


def test_batch_tune(pkg):
    wls = cases(n=3)
    a = make_batch(pkg, wls)
    g, k, ms = a.tune(2)
    assert g in (4, 8, 16, 32, 64) and k in (1, 2, 4, 8) and ms > 0
    assert a.steps == 80
    a.step(1)
    b = make_batch(pkg, wls)
    b.step(81)
    for c in range(len(wls)):
        for x, y in zip(state(a, c), state(b, c)):
            assert np.array_equal(x, y)


def test_batch_case_vs_oracle(pkg, oracle_mod):
    """Case 1 of the batch against the FP64 oracle after three steps, within
    the single-lattice FP32 tolerances (populations 2e-6 absolute; force 2e-6
    per link plus 1e-5 relative)."""
    wls = cases()
    wls = [H.with_margin(oracle_mod, wl) for wl in wls]
    b = make_batch(pkg, wls)
    b.step(3)
    wl = wls[1]
    orc = H.make_oracle(oracle_mod, wl)
    orc.set_particles(H.oracle_particles(oracle_mod, wl))
    orc.step(3)
    own = orc.owner()
    fg = b.populations(1).cpu().numpy()
    assert np.abs(fg - orc.populations())[:, own < 0].max() <= 2e-6
    Fg, _ = b.forces(1)
    Fo, _ = orc.forces()
    nl = orc.counters()["nlinks"]
    assert np.abs(Fg - Fo).max() <= 2e-6 * nl + 1e-5 * np.abs(Fo).max()


def test_batch_rejects(pkg):
    wls = cases(n=2)
    bad = [cfg_kw(wl) for wl in wls]
    bad[1]["storage"] = "f64"
    with pytest.raises(pkg.LbmError):
        pkg.Batch(bad)
    bad = [cfg_kw(wl) for wl in wls]
    bad[0]["n_sub"] = 10
    with pytest.raises(pkg.LbmError):
        pkg.Batch(bad)
    b = pkg.Batch([cfg_kw(wl) for wl in wls])
    p = dict(wls[0]["particles"][0])
    p["fixed"] = 0
    with pytest.raises(pkg.LbmError) as e:
        b.set_particles(0, H.gpu_particles(pkg, dict(particles=[p])))
    assert e.value.code == -1
