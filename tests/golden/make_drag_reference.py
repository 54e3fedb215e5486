"""Writes drag_reference.json: the FP64 oracle's hydrodynamic force and
torque on the fixed metaball of workloads.drag_case() after its steps (the
expected value of the reduced-precision drag check).  Calls only the oracle.

    python tests/golden/make_drag_reference.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2206_11634_gb300 import workloads as W  # noqa: E402
from tests import _helpers as H  # noqa: E402


def main():
    wl = H.with_margin(O, W.drag_case())
    orc = H.make_oracle(O, wl)
    orc.set_particles(H.oracle_particles(O, wl))
    hist = []
    for k in range(wl["steps"]):
        orc.step(1)
        if (k + 1) % 100 == 0:
            F, T = orc.forces()
            hist.append({"step": k + 1, "F": F[0].tolist(), "T": T[0].tolist()})
    F, T = orc.forces()
    out = {"case": wl["name"], "steps": wl["steps"], "x": wl["particles"][0]["x"].tolist(),
           "F": F[0].tolist(), "T": T[0].tolist(), "history": hist,
           "source": "FP64 oracle (oracle/lbm_oracle.c), tests/golden/make_drag_reference.py"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "drag_reference.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["F"])


if __name__ == "__main__":
    main()
