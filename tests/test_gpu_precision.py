"""Drag of the reduced-precision storage forms against the FP64 oracle.

The case is workloads.drag_case(): a fixed four-control-point metaball in a
periodic 48^3 box, flow driven by a Guo body force, 1000 steps from rest.
The expected force history is the FP64 oracle's (tests/golden/
drag_reference.json, written by tests/golden/make_drag_reference.py).

The sweep computes in offset form (g = f - w rho0), so rounding is relative
to the flow signal, not to w rho0; at this low speed (|u| ~ 1e-3) that is
what lets FP32 hold the drag to ~1e-5 (computing with f itself gave 2e-3).

Tolerances on the relative error of the drag F_x:
- FP32 storage and collision: 1e-4 (measured 1.5e-5);
- FP16 offsets (11 significant bits of s = f/w - rho0): 1e-3, the target
  for the reduced-precision form;
- BF16 offsets (8 significant bits, rounding eight times coarser than
  FP16): 3e-2 (measured 1.3e-2); BF16 does not reach the 1e-3 target.
"""
import json
import os

import numpy as np
import pytest

from tests import _helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts
    pytest.skip("no CUDA device", allow_module_level=True)

REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "drag_reference.json")


@pytest.fixture(scope="module")
def pkg():
    from paper_2206_11634_gb300 import build as b
    b.build()
    import paper_2206_11634_gb300 as p
    return p


@pytest.mark.parametrize("storage,tol", [("f32", 1e-4), ("f16", 1e-3), ("bf16", 3e-2)])
def test_drag_vs_oracle(pkg, storage, tol):
    from paper_2206_11634_gb300 import workloads as W
    ref = json.load(open(REF))
    wl = W.drag_case(storage)
    assert ref["case"] == wl["name"] and ref["steps"] == wl["steps"]
    wl["particles"][0]["x"] = np.array(ref["x"])
    gpu = H.make_gpu(pkg, wl)
    gpu.set_particles(H.gpu_particles(pkg, wl))
    done = 0
    worst = 0.0
    for h in ref["history"]:
        gpu.step(h["step"] - done)
        done = h["step"]
        F, _ = gpu.forces()
        rel = abs(F[0, 0] - h["F"][0]) / abs(h["F"][0])
        worst = max(worst, rel)
        # the cross-flow components are ~100x smaller; bound them on the drag's scale
        assert np.abs(F[0, 1:] - np.array(h["F"][1:])).max() <= tol * abs(h["F"][0])
    print(f"{storage}: worst relative drag error {worst:.2e}")
    assert worst <= tol
