"""The two-particle settling run of §4 (drafting, kissing, tumbling), on the
GPU, at the paper's box (150 x 150 x 250 nodes at 1 mm), densities (1200 and
927 kg/m^3), gravity and start positions (220 and 205 nodes above the
bottom, the lower particle 2 nodes off the centre line), tau 0.56 (the
paper's viscosity gives 0.545, where the scheme diverges; see the workload).

The paper compares with no data here, so the check is qualitative, on the
three phases that define the phenomenon:
- drafting: in the leader's wake the trailing particle falls faster;
- kissing: the two come within touching distance (centres within 1.1
  volume-equivalent diameters, 14.65 nodes);
- tumbling: the pair turns over: the trailing particle passes below the
  leader, the two separated sideways.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

D_EQ = 2.0 * 7.325  # volume-equivalent diameter of both shapes (1648 cells)


@pytest.fixture(scope="module")
def pkg():
    from paper_2206_11634_gb300 import build as b
    b.build()
    import paper_2206_11634_gb300 as p
    return p


def _run(pkg, wl, steps, every):
    lat = pkg.Lattice(wl["nx"], wl["ny"], wl["nz"], periodic=wl["periodic"], lattice=19, storage=wl["storage"],
                      n_sub=wl["n_sub"], max_particles=2, tau=wl["tau"], gravity=wl["gravity"], force=wl["force"],
                      kn=wl["kn"], eta_n=wl["eta_n"], kt=wl["kt"], eta_t=wl["eta_t"], mu_s=wl["mu_s"],
                      c_tol=wl["c_tol"])
    lat.set_particles([pkg.make_particle(p["cp"], p["K"], p["x"], q=p["q"], Rs=p["Rs"], density=p["density"])
                       for p in wl["particles"]])
    xs, vs = [], []
    for _ in range(0, steps + 1, every):
        st = lat.particles()
        xs.append([p["x"] for p in st])
        vs.append([p["v"] for p in st])
        lat.step(every)
    lat.check()
    return np.array(xs), np.array(vs)


@pytest.mark.parametrize("shape", ["metaball", "sphere"])
def test_dkt_draft_kiss_tumble(pkg, shape):
    from paper_2206_11634_gb300 import workloads as W
    wl = W.dkt(shape)
    x, v = _run(pkg, wl, 5500, 250)  # particle 0 starts above (trails), 1 below (leads)
    # drafting: while still above the leader, the trailing particle falls
    # more than 5 % faster, and the vertical gap closes from its 15 nodes
    above = x[:, 0, 2] > x[:, 1, 2] + 5.0
    ratio = np.where(above, v[:, 0, 2] / np.minimum(v[:, 1, 2], -1e-12), 0.0)
    assert ratio.max() > 1.05, ratio
    assert x[10, 0, 2] - x[10, 1, 2] < 14.0, x[10]  # 2500 steps
    # kissing: centres within touching distance
    dist = np.linalg.norm(x[:, 0] - x[:, 1], axis=1)
    assert dist.min() < 1.1 * D_EQ, dist.min()
    # tumbling: the trailing particle ends below the leader, side by side
    assert x[-1, 0, 2] < x[-1, 1, 2], x[-1]
    assert abs(x[-1, 0, 0] - x[-1, 1, 0]) > 5.0, x[-1]
    # both still above the floor and in the box
    assert np.all(x[:, :, 2] > 10.0) and np.all((x[:, :, :2] > 10.0) & (x[:, :, :2] < 140.0))


def test_dkt_window_against_oracle(pkg, oracle_mod):
    """A 50-step window of the metaball run compared with the FP64 oracle,
    re-synchronised when the pair approaches the kiss (centres within 1.3
    equivalent diameters, no contact yet): the oracle takes the GPU's
    populations, node owners and particle states, then both step 50 times.
    The hydrodynamic force on each particle agrees every step within 2e-3 of
    its size plus 1e-4 of the largest (FP32 sums over ~1500 links of values
    that differ by ~1e-6), and after the window positions within 2e-4 lu,
    velocities within 2e-5 and angular velocities within 5e-5."""
    from paper_2206_11634_gb300 import workloads as W
    wl = W.dkt("metaball")
    lat = pkg.Lattice(wl["nx"], wl["ny"], wl["nz"], periodic=wl["periodic"], lattice=19, storage=wl["storage"],
                      n_sub=wl["n_sub"], max_particles=2, tau=wl["tau"], gravity=wl["gravity"], force=wl["force"],
                      kn=wl["kn"], eta_n=wl["eta_n"], kt=wl["kt"], eta_t=wl["eta_t"], mu_s=wl["mu_s"],
                      c_tol=wl["c_tol"])
    lat.set_particles([pkg.make_particle(p["cp"], p["K"], p["x"], q=p["q"], Rs=p["Rs"], density=p["density"])
                       for p in wl["particles"]])
    for _ in range(40):
        lat.step(100)
        st = lat.particles()
        if np.linalg.norm(st[0]["x"] - st[1]["x"]) < 1.3 * D_EQ:
            break
    else:
        raise AssertionError("the pair did not approach")
    Fc, _ = lat.contact_forces()
    assert not Fc.any()
    orc = oracle_mod.Oracle(wl["nx"], wl["ny"], wl["nz"], Q=19, periodic=wl["periodic"], tau=wl["tau"],
                            n_sub=wl["n_sub"], gravity=wl["gravity"], force=wl["force"], kn=wl["kn"],
                            eta_n=wl["eta_n"], kt=wl["kt"], eta_t=wl["eta_t"], mu_s=wl["mu_s"], c_tol=wl["c_tol"])
    # the GPU's particle states, with its mass properties (both sides then use
    # the same values and frames)
    orc.set_particles([oracle_mod.make_particle(s["cp"], s["K"], s["x"], q=s["q"], v=s["v"], w=s["w"], Rs=s["Rs"],
                                                density=s["density"], mass=s["mass"], inertia=s["inertia"])
                       for s in st])
    orc.set_owner(lat.flags().cpu().numpy().astype(np.int32) - 1)
    orc.set_populations(lat.populations().cpu().numpy())
    for _ in range(50):
        lat.step(1)
        orc.step(1)
        Fg, _ = lat.forces()
        Fo, _ = orc.forces()
        assert np.all(np.abs(Fg - Fo) <= 2e-3 * np.abs(Fo) + 1e-4 * np.abs(Fo).max()), (Fg, Fo)
    for sg, so in zip(lat.particles(), orc.get_particles()):
        assert np.abs(sg["x"] - so["x"]).max() < 2e-4, (sg["x"], so["x"])
        assert np.abs(sg["v"] - so["v"]).max() < 2e-5, (sg["v"], so["v"])
        assert np.abs(sg["w"] - so["w"]).max() < 5e-5, (sg["w"], so["w"])
