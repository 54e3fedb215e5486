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
