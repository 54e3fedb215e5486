"""ctypes front end of the FP64 CPU oracle (oracle/lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle shares no
code with the CUDA library and is never called by it.

Everything is plain double precision; arrays are numpy.  Populations use the
layout f[i, z, y, x] (direction-major, x fastest), the same structure-of-arrays
order the library's test hooks expose, so the two can be compared directly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

MAXCP = 16


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction so x86 and Arm
    round identically).  Returns the path of the shared object."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("Q", C.c_int),
        ("periodic", C.c_int * 3),
        ("n_sub", C.c_int),
        ("vibb", C.c_int),
        ("missing_force", C.c_int),
        ("nthreads", C.c_int),
        ("q_exact", C.c_int),
        ("tau", C.c_double), ("rho0", C.c_double), ("c0", C.c_double),
        ("u0", C.c_double * 3),
        ("force", C.c_double * 3),
        ("gravity", C.c_double * 3),
        ("kn", C.c_double), ("eta_n", C.c_double), ("kt", C.c_double),
        ("eta_t", C.c_double), ("mu_s", C.c_double), ("c_tol", C.c_double),
        ("mass_spacing", C.c_double),
    ]


class Particle(C.Structure):
    _fields_ = [
        ("ncp", C.c_int), ("fixed", C.c_int),
        ("cp", (C.c_double * 3) * MAXCP),
        ("K", C.c_double * MAXCP),
        ("Rs", C.c_double), ("density", C.c_double), ("mass", C.c_double),
        ("inertia", C.c_double * 9),
        ("x", C.c_double * 3), ("q", C.c_double * 4),
        ("v", C.c_double * 3), ("w", C.c_double * 3),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(Config)]
        L.orc_destroy.argtypes = [P]
        L.orc_set_particles.argtypes = [P, C.POINTER(Particle), C.c_int]
        L.orc_set_particles.restype = C.c_int
        L.orc_get_particles.argtypes = [P, C.POINTER(Particle)]
        L.orc_step.argtypes = [P, C.c_int]
        L.orc_classify.argtypes = [P, ip]
        L.orc_freeze_flags.argtypes = [P, C.c_int]
        L.orc_metaball.argtypes = [P, C.c_int, dp]
        L.orc_metaball.restype = C.c_double
        L.orc_metaball_dd.argtypes = [P, C.c_int, dp, dp, dp, dp]
        L.orc_q_linear.argtypes = [P, C.c_int, dp, dp]
        L.orc_q_linear.restype = C.c_double
        L.orc_q_newton.argtypes = [P, C.c_int, dp, dp, C.c_double, C.c_int, dp]
        L.orc_q_newton.restype = C.c_int
        L.orc_lattice.argtypes = [P, ip, ip, dp, ip]
        L.orc_equilibrium.argtypes = [P, C.c_double, dp, dp]
        for name in ("orc_get_populations", "orc_set_populations"):
            getattr(L, name).argtypes = [P, dp]
        L.orc_get_owner.argtypes = [P, ip]
        L.orc_set_owner.argtypes = [P, ip]
        L.orc_get_fields.argtypes = [P, dp, dp]
        L.orc_get_forces.argtypes = [P, dp, dp]
        L.orc_get_contact_forces.argtypes = [P, dp, dp]
        L.orc_counters.argtypes = [P, C.POINTER(C.c_long), ip, ip]
        L.orc_min_margin.argtypes = [P]
        L.orc_min_margin.restype = C.c_double
        L.orc_mass_properties.argtypes = [C.POINTER(Particle), C.c_double, C.c_double]
        L.orc_pair_geometry.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.orc_pair_geometry.restype = C.c_int
        L.orc_wall_geometry.argtypes = [P, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.orc_wall_geometry.restype = C.c_int
        L.orc_vibb_unknown.argtypes = [P, C.c_int, C.c_double, dp, dp, dp]
        L.orc_vibb_unknown.restype = C.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _vec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


DEFAULTS = dict(Q=19, periodic=(0, 0, 0), n_sub=0, vibb=1, missing_force=1, nthreads=0, q_exact=0,
                tau=0.8, rho0=1.0, c0=1.0, u0=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0),
                gravity=(0.0, 0.0, 0.0), kn=0.0, eta_n=0.0, kt=0.0, eta_t=0.0, mu_s=0.0,
                c_tol=1e-6, mass_spacing=0.5)


def make_config(nx: int, ny: int, nz: int, **kw) -> Config:
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError(f"unknown oracle config keys {sorted(unknown)}")
    d.update(kw)
    c = Config()
    c.nx, c.ny, c.nz = nx, ny, nz
    for k, v in d.items():
        f = getattr(c, k)
        if isinstance(f, C.Array):
            for i, x in enumerate(v):
                f[i] = x
        else:
            setattr(c, k, v)
    return c


def make_particle(cp: Sequence[Sequence[float]], K: Sequence[float], x, *, q=(1, 0, 0, 0), v=(0, 0, 0),
                  w=(0, 0, 0), Rs=0.0, density=1.0, mass=0.0, inertia=None, fixed=0) -> Particle:
    p = Particle()
    cp = np.asarray(cp, dtype=np.float64).reshape(-1, 3)
    if not 1 <= len(cp) <= MAXCP or len(K) != len(cp):
        raise ValueError("1..16 control points with one weight each")
    p.ncp = len(cp)
    p.fixed = int(fixed)
    for k in range(len(cp)):
        for a in range(3):
            p.cp[k][a] = cp[k, a]
        p.K[k] = K[k]
    p.Rs, p.density, p.mass = Rs, density, mass
    if inertia is not None:
        for i, val in enumerate(np.asarray(inertia, dtype=np.float64).reshape(9)):
            p.inertia[i] = val
    for a in range(3):
        p.x[a], p.v[a], p.w[a] = x[a], v[a], w[a]
    for a in range(4):
        p.q[a] = q[a]
    return p


def particle_dict(p: Particle) -> dict:
    n = p.ncp
    return dict(ncp=n, fixed=p.fixed, cp=np.array([[p.cp[k][a] for a in range(3)] for k in range(n)]),
                K=np.array([p.K[k] for k in range(n)]), Rs=p.Rs, density=p.density, mass=p.mass,
                inertia=np.array(list(p.inertia)).reshape(3, 3), x=np.array(list(p.x)),
                q=np.array(list(p.q)), v=np.array(list(p.v)), w=np.array(list(p.w)))


class Oracle:
    """One oracle simulation (lattice, populations, particles)."""

    def __init__(self, nx: int, ny: int, nz: int, **kw):
        self.cfg = make_config(nx, ny, nz, **kw)
        self.L = lib()
        self.h = self.L.orc_create(C.byref(self.cfg))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        Q = C.c_int()
        e = np.zeros(19 * 3, dtype=np.int32)
        w = np.zeros(19)
        opp = np.zeros(19, dtype=np.int32)
        self.L.orc_lattice(self.h, C.byref(Q), _ip(e), _dp(w), _ip(opp))
        self.Q = Q.value
        self.e = e[: 3 * self.Q].reshape(self.Q, 3).copy()
        self.w = w[: self.Q].copy()
        self.opp = opp[: self.Q].copy()
        self.np = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    # particles -------------------------------------------------------------
    def set_particles(self, particles: Iterable[Particle]):
        arr_t = Particle * max(1, len(list(particles)))
        plist = list(particles)
        arr = arr_t(*plist)
        if self.L.orc_set_particles(self.h, arr, len(plist)) != 0:
            raise ValueError("oracle rejected the particles")
        self.np = len(plist)

    def get_particles(self) -> list[dict]:
        arr = (Particle * max(1, self.np))()
        self.L.orc_get_particles(self.h, arr)
        return [particle_dict(arr[j]) for j in range(self.np)]

    # stepping --------------------------------------------------------------
    def step(self, n: int = 1):
        self.L.orc_step(self.h, int(n))

    # state access ----------------------------------------------------------
    def populations(self) -> np.ndarray:
        out = np.empty((self.Q,) + self.shape)
        self.L.orc_get_populations(self.h, _dp(out))
        return out

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((self.Q,) + self.shape)
        self.L.orc_set_populations(self.h, _dp(f))

    def owner(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.int32)
        self.L.orc_get_owner(self.h, _ip(out))
        return out

    def set_owner(self, own: np.ndarray):
        own = np.ascontiguousarray(own, dtype=np.int32).reshape(self.shape)
        self.L.orc_set_owner(self.h, _ip(own))

    def freeze_flags(self, on: bool = True) -> None:
        """Classify the current particles once and keep those node flags
        (q still follows the particles); on=False releases them."""
        self.L.orc_freeze_flags(self.h, int(on))

    def classify(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.int32)
        self.L.orc_classify(self.h, _ip(out))
        return out

    def fields(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        self.L.orc_get_fields(self.h, _dp(rho), _dp(u))
        return rho, u

    def forces(self):
        F = np.zeros((max(1, self.np), 3))
        T = np.zeros((max(1, self.np), 3))
        self.L.orc_get_forces(self.h, _dp(F), _dp(T))
        return F[: self.np], T[: self.np]

    def contact_forces(self):
        F = np.zeros((max(1, self.np), 3))
        T = np.zeros((max(1, self.np), 3))
        self.L.orc_get_contact_forces(self.h, _dp(F), _dp(T))
        return F[: self.np], T[: self.np]

    def counters(self) -> dict:
        st, nr, nl = C.c_long(), C.c_int(), C.c_int()
        self.L.orc_counters(self.h, C.byref(st), C.byref(nr), C.byref(nl))
        return dict(step=st.value, nrefill=nr.value, nlinks=nl.value)

    # geometry pieces ---------------------------------------------------------
    def metaball(self, j: int, x) -> float:
        return self.L.orc_metaball(self.h, j, _dp(_vec(x)))

    def metaball_dd(self, j: int, x):
        M = np.zeros(1)
        g = np.zeros(3)
        H = np.zeros(9)
        self.L.orc_metaball_dd(self.h, j, _dp(_vec(x)), _dp(M), _dp(g), _dp(H))
        return M[0], g, H.reshape(3, 3)

    def q_linear(self, j: int, xf, d) -> float:
        return self.L.orc_q_linear(self.h, j, _dp(_vec(xf)), _dp(_vec(d)))

    def q_newton(self, j: int, xf, d, tol=1e-7, maxit=100):
        q = np.zeros(1)
        it = self.L.orc_q_newton(self.h, j, _dp(_vec(xf)), _dp(_vec(d)), tol, maxit, _dp(q))
        return q[0], it

    def vibb_unknown(self, i: int, q: float, fplus_f, fplus_ff, uw) -> float:
        """The unknown f_i(x_f, t+1) of one particle link from raw inputs
        (halfway bounce-back when ``fplus_ff`` is None)."""
        fff = None if fplus_ff is None else _dp(_vec(fplus_ff))
        return self.L.orc_vibb_unknown(self.h, i, q, _dp(_vec(fplus_f)), fff, _dp(_vec(uw)))

    def equilibrium(self, rho: float, u) -> np.ndarray:
        out = np.zeros(self.Q)
        self.L.orc_equilibrium(self.h, rho, _dp(_vec(u)), _dp(out))
        return out

    def min_margin(self) -> float:
        return self.L.orc_min_margin(self.h)

    def pair_geometry(self, i: int, j: int, xm_start=None):
        xm = np.zeros(3)
        delta = np.zeros(1)
        n = np.zeros(3)
        xcp = np.zeros(3)
        start = None if xm_start is None else _dp(_vec(xm_start))
        hit = self.L.orc_pair_geometry(self.h, i, j, start, _dp(xm), _dp(delta), _dp(n), _dp(xcp))
        return bool(hit), delta[0], n, xcp, xm

    def wall_geometry(self, j: int, wall: int, start=None):
        xcw = np.zeros(3)
        delta = np.zeros(1)
        n = np.zeros(3)
        xcp = np.zeros(3)
        st = None if start is None else _dp(_vec(start))
        hit = self.L.orc_wall_geometry(self.h, j, wall, st, _dp(xcw), _dp(delta), _dp(n), _dp(xcp))
        return bool(hit), delta[0], n, xcp, xcw


def mass_properties(p: Particle, c0: float = 1.0, spacing: float = 0.5) -> Particle:
    q = Particle()
    C.pointer(q)[0] = p
    lib().orc_mass_properties(C.byref(q), c0, spacing)
    return q

