"""Helpers shared by the parity tests: one workload description feeds both the
CPU oracle and the CUDA library through their own constructors."""
from __future__ import annotations

import numpy as np

PHYS_KEYS = ("tau", "n_sub", "gravity", "force", "kn", "eta_n", "kt", "eta_t", "mu_s", "c_tol")


def oracle_particles(oracle_mod, wl):
    out = []
    for p in wl["particles"]:
        kw = dict(q=p["q"], v=p["v"], w=p["w"], Rs=p["Rs"], density=p["density"], mass=p["mass"], fixed=p["fixed"])
        if p.get("inertia") is not None:
            kw["inertia"] = p["inertia"]
        out.append(oracle_mod.make_particle(p["cp"], p["K"], p["x"], **kw))
    return out


def gpu_particles(pkg, wl):
    out = []
    for p in wl["particles"]:
        kw = dict(q=p["q"], v=p["v"], w=p["w"], Rs=p["Rs"], density=p["density"], mass=p["mass"], fixed=p["fixed"])
        if p.get("inertia") is not None:
            kw["inertia"] = p["inertia"]
        out.append(pkg.make_particle(p["cp"], p["K"], p["x"], **kw))
    return out


def make_oracle(oracle_mod, wl, Q=19, **over):
    kw = {k: wl[k] for k in PHYS_KEYS}
    kw.update(periodic=tuple(wl["periodic"]), Q=Q)
    kw.update(wl.get("extra_oracle", {}))
    kw.update(over)
    o = oracle_mod.Oracle(wl["nx"], wl["ny"], wl["nz"], **kw)
    return o


def make_gpu(pkg, wl, Q=19, storage=None, **over):
    kw = {k: wl[k] for k in PHYS_KEYS}
    kw.update(periodic=tuple(wl["periodic"]), lattice=Q, storage=storage or wl["storage"],
              max_particles=max(1, len(wl["particles"])))
    kw.update(over)
    return pkg.Lattice(wl["nx"], wl["ny"], wl["nz"], **kw)


def with_margin(oracle_mod, wl, rng=None, min_margin=1e-9, tries=20):
    """Shift particle positions by tiny amounts until no node of any search
    box lies within min_margin (relative) of a surface, as the oracle
    evaluates it.  Returns the (possibly shifted) workload."""
    rng = rng or np.random.default_rng(0)
    for _ in range(tries):
        o = make_oracle(oracle_mod, wl)
        o.set_particles(oracle_particles(oracle_mod, wl))
        if not wl["particles"] or o.min_margin() > min_margin:
            return wl
        for p in wl["particles"]:
            p["x"] = p["x"] + rng.uniform(-1e-4, 1e-4, 3)
    raise RuntimeError("could not move the surfaces away from the nodes")


def fixed_mass(wl, mass=50.0, inertia=500.0):
    """Give every particle explicit mass properties (both sides then use the
    same values and frames)."""
    for p in wl["particles"]:
        p["mass"] = mass
        p["inertia"] = np.eye(3) * inertia
    return wl


def fluid_mask_from_flags(flags):
    return np.asarray(flags) == 0


# --------------------------------------------------------------------------
# drag gradient (flags frozen): the oracle's objective for finite differences
# --------------------------------------------------------------------------
def adjoint_particle_kw(case, cp_world, K):
    """A fixed particle with identity orientation whose world control points
    are cp_world (body frame = cp_world - x)."""
    x = np.asarray(case["x"], dtype=np.float64)
    return dict(cp=np.asarray(cp_world, dtype=np.float64) - x, K=np.asarray(K, dtype=np.float64), x=x,
                q=(1.0, 0.0, 0.0, 0.0), fixed=1, mass=1.0, inertia=np.eye(3))


def oracle_drag_J(oracle_mod, case, cp_world, K, base=None):
    """Mean F_x over the last W of T steps of the FP64 oracle, with the node
    flags classified from `base` (cp_world, K) and frozen while the particle
    has (cp_world, K); missing force points off (with frozen flags and one
    particle every crossing link is an Eq. (28) link)."""
    base = base or (case["cp_world"], case["K"])
    o = oracle_mod.Oracle(case["nx"], case["ny"], case["nz"], periodic=(1, 1, 1), tau=case["tau"],
                          u0=tuple(case["u0"]), force=tuple(case["force"]), missing_force=0)
    kw = adjoint_particle_kw(case, *base)
    o.set_particles([oracle_mod.make_particle(kw.pop("cp"), kw.pop("K"), kw.pop("x"), **kw)])
    o.freeze_flags(True)
    kw = adjoint_particle_kw(case, cp_world, K)
    o.set_particles([oracle_mod.make_particle(kw.pop("cp"), kw.pop("K"), kw.pop("x"), **kw)])
    T, W = case["T"], case["W"]
    o.step(T - W)
    J = 0.0
    for _ in range(W):
        o.step(1)
        F, _ = o.forces()
        J += F[0, 0]
    return J / W, o

