"""GPU drag gradient (include/lbm_adjoint.h): the hand-written discrete
adjoint of the sweep, the interpolated bounce-back and the momentum exchange,
flags frozen, against central finite differences of the FP64 oracle with the
same frozen flags (tests/test_oracle_adjoint.py pins that reference).

Tolerances:
- J (mean drag over the window) of the FP32 forward run: 1e-4 relative to the
  FP64 oracle (offset-form FP32 keeps the drag to ~1e-5, see
  tests/test_gpu_precision.py);
- gradient: every component within 1e-4 of the largest one, the target for
  the adjoint (measured 2e-6: the FP32 adjoint differentiates the FP32
  forward run, whose drag differs from the FP64 one by ~1e-5; the central
  differences use h = 1e-5, where the oracle's rounding noise is ~1e-11
  relative and q crosses no branch point);
- the autograd wrapper returns the library's gradient (to the run-to-run
  spread of the adjoint's FP32 atomic scatter, ~1e-7 of the largest
  component; the test allows 1e-5).
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


def small_case():
    from paper_2206_11634_gb300 import workloads as W
    return W.adjoint_case(n=32, ncp=3, T=80, W=20)


def engine(pkg, case):
    from paper_2206_11634_gb300.adjoint import AdjointDrag
    kw = H.adjoint_particle_kw(case, case["cp_world"], case["K"])
    p = pkg.make_particle(kw.pop("cp"), kw.pop("K"), kw.pop("x"), **kw)
    return AdjointDrag(case["nx"], case["ny"], case["nz"], particle=p, T=case["T"], W=case["W"], tau=case["tau"],
                       u0=case["u0"], force=case["force"])


def oracle_fd(oracle_mod, case, h_pos=1e-5, h_rel=1e-5):
    cp, K = case["cp_world"], case["K"]
    g_cp = np.zeros_like(cp)
    g_K = np.zeros_like(K)
    for c in range(len(K)):
        for a in range(3):
            e = np.zeros_like(cp)
            e[c, a] = h_pos
            Jp, _ = H.oracle_drag_J(oracle_mod, case, cp + e, K)
            Jm, _ = H.oracle_drag_J(oracle_mod, case, cp - e, K)
            g_cp[c, a] = (Jp - Jm) / (2 * h_pos)
        e = np.zeros_like(K)
        e[c] = h_rel * K[c]
        Jp, _ = H.oracle_drag_J(oracle_mod, case, cp, K + e)
        Jm, _ = H.oracle_drag_J(oracle_mod, case, cp, K - e)
        g_K[c] = (Jp - Jm) / (2 * e[c])
    return g_cp, g_K


def test_forward_matches_oracle(pkg, oracle_mod):
    case = small_case()
    eng = engine(pkg, case)
    J = eng.forward_np(case["cp_world"], case["K"])
    Jo, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"], case["K"])
    print("J", J, Jo, eng.info())
    assert abs(J - Jo) <= 1e-4 * abs(Jo)


def test_gradient_matches_oracle_fd(pkg, oracle_mod):
    case = small_case()
    eng = engine(pkg, case)
    eng.forward_np(case["cp_world"], case["K"])
    g_cp, g_K = eng.backward_np()
    f_cp, f_K = oracle_fd(oracle_mod, case)
    # compare d/dK in the same units as d/dx: dJ/d(ln K)
    a = np.concatenate([g_cp.ravel(), g_K * case["K"]])
    b = np.concatenate([f_cp.ravel(), f_K * case["K"]])
    err = np.abs(a - b).max() / np.abs(b).max()
    print("adjoint", a, "\nfd     ", b, "\nrel err", err)
    assert err <= 1e-4


def test_autograd_wrapper(pkg):
    case = small_case()
    eng = engine(pkg, case)
    cp = torch.tensor(case["cp_world"], dtype=torch.float64, requires_grad=True)
    K = torch.tensor(case["K"], dtype=torch.float64, requires_grad=True)
    J = eng(cp, K)
    J.backward()
    g_cp, g_K = eng.backward_np()
    # a second backward run differs only by the order of the adjoint's FP32
    # atomic scatter (~1e-7 of the largest component)
    scale = max(np.abs(g_cp).max(), np.abs(g_K * case["K"]).max())
    assert np.abs(cp.grad.numpy() - g_cp).max() <= 1e-5 * scale
    assert np.abs((K.grad.numpy() - g_K) * case["K"]).max() <= 1e-5 * scale
    assert np.isclose(J.item(), eng.forward_np(case["cp_world"], case["K"]), rtol=0, atol=0)


def test_full_size_gradient(pkg, oracle_mod):
    """Workload 4 at its size (96^3, six control points, T = 500, W = 100,
    checkpoints every 23 steps): dJ/dK_0 against the oracle's central
    difference (1e-4 relative), and the whole gradient against a directional
    central difference of the GPU forward run along it.  That difference takes
    h = 2e-3 (J is piecewise smooth in the shape: q has a branch point at 1/2
    and clamps at 0 and 1, and a larger step moves some links across them),
    where the FP32 forward's noise (~1e-6 of J) is ~1e-3 of the change: 1e-2."""
    from paper_2206_11634_gb300 import workloads as W
    case = W.adjoint_case()
    eng = engine(pkg, case)
    assert eng.info()["checkpoint_every"] == 23
    J0 = eng.forward_np(case["cp_world"], case["K"])
    g_cp, g_K = eng.backward_np()
    assert np.all(np.isfinite(g_cp)) and np.all(np.isfinite(g_K))
    hK = 1e-5 * case["K"][0]
    e = np.zeros_like(case["K"])
    e[0] = hK
    Jp, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"], case["K"] + e)
    Jm, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"], case["K"] - e)
    fK = (Jp - Jm) / (2 * hK)
    print("dJ/dK0", g_K[0], fK)
    assert abs(g_K[0] - fK) <= 1e-4 * abs(fK)
    v = np.concatenate([g_cp.ravel(), g_K * case["K"]])
    d = v / np.linalg.norm(v)
    h = 2e-3
    n3 = 3 * len(case["K"])
    cp_p = case["cp_world"] + h * d[:n3].reshape(-1, 3)
    cp_m = case["cp_world"] - h * d[:n3].reshape(-1, 3)
    K_p = case["K"] * (1 + h * d[n3:])
    K_m = case["K"] * (1 - h * d[n3:])
    fd = (eng.forward_np(cp_p, K_p) - eng.forward_np(cp_m, K_m)) / (2 * h)
    print("J", J0, "directional", fd, np.linalg.norm(v))
    assert abs(fd - np.linalg.norm(v)) <= 1e-2 * np.linalg.norm(v)
