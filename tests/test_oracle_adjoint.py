"""The finite-difference reference of the drag gradient: the FP64 oracle with
frozen node flags (q follows the shape, the link set does not).

Pins, independent of the GPU path:
- frozen flags stay put while the shape moves, and the drag responds;
- mirror symmetry: for a sphere at the centre of a periodic box with the flow
  along x, moving the sphere along y or z changes the drag only at second
  order (the y -> -y mirror maps J(y + h) onto J(y - h)), so the central
  differences in y and z vanish to rounding while the one in x need not;
- a larger sphere (larger K) feels more drag: dJ/dK > 0.
"""
import numpy as np
import pytest

from tests import _helpers as H


def sphere_case(n=16, T=24, W=8):
    c = n / 2.0 - 0.5
    return dict(nx=n, ny=n, nz=n, tau=0.8, u0=(0.02, 0.0, 0.0), force=(2e-6, 0.0, 0.0), T=T, W=W,
                x=np.full(3, c), cp_world=np.array([[c, c, c]]), K=np.array([12.25]))


def test_frozen_flags_hold(oracle_mod):
    case = sphere_case()
    J0, o0 = H.oracle_drag_J(oracle_mod, case, case["cp_world"], case["K"])
    moved = case["cp_world"] + np.array([[0.3, 0.0, 0.0]])
    J1, o1 = H.oracle_drag_J(oracle_mod, case, moved, case["K"])
    assert np.array_equal(o0.owner(), o1.owner())
    assert abs(J1 - J0) > 1e-9 * abs(J0)


def test_mirror_symmetry_of_the_gradient(oracle_mod):
    case = sphere_case()
    h = 1e-4
    d = []
    for a in range(3):
        e = np.zeros((1, 3))
        e[0, a] = h
        Jp, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"] + e, case["K"])
        Jm, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"] - e, case["K"])
        d.append((Jp - Jm) / (2 * h))
    hK = 1e-4 * case["K"][0]
    Jp, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"], case["K"] + hK)
    Jm, _ = H.oracle_drag_J(oracle_mod, case, case["cp_world"], case["K"] - hK)
    dK = (Jp - Jm) / (2 * hK)
    scale = abs(dK) * case["K"][0]  # drag change per unit relative change in K
    assert dK > 0
    assert abs(d[1]) < 1e-8 * scale and abs(d[2]) < 1e-8 * scale, (d, scale)
