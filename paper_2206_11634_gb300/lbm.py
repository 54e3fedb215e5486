"""Thin Python binding of the C ABI in include/lbm_metaball.h.

Argument marshalling only: every step of the lattice sweep runs in the CUDA
library (paper_2206_11634_gb300/_lib/liblbmmb.so).  PyTorch provides the
device workspace and the CUDA stream.  There is no CPU fallback: when the
library is missing or no GPU is present the constructor raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblbmmb.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "lbm_metaball.h")

MAX_CP = 16
MAX_PER_BRICK = 16
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
# lbm_config.dem_mode: FP64 rigid-body integrator (default), compensated FP32
# integrator, FP64 contact geometry as well
DEM_MODE = {"fp64": 0, "fp32": 1, "fp64_all": 2}
STATUS = {0: "LBM_OK", -1: "LBM_ERR_BAD_ARG", -2: "LBM_ERR_WS_TOO_SMALL", -3: "LBM_ERR_CAPACITY",
          -4: "LBM_ERR_DIVERGED", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_CUDA"}


class LbmConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("lattice", C.c_int32), ("storage", C.c_int32),
        ("periodic", C.c_int32 * 3),
        ("n_sub", C.c_int32), ("vibb", C.c_int32), ("missing_force", C.c_int32),
        ("max_particles", C.c_int32),
        ("dem_mode", C.c_int32), ("q_exact", C.c_int32),
        ("tau", C.c_double), ("rho0", C.c_double), ("c0", C.c_double),
        ("u0", C.c_double * 3), ("force", C.c_double * 3), ("gravity", C.c_double * 3),
        ("kn", C.c_double), ("eta_n", C.c_double),
        ("kt", C.c_double), ("eta_t", C.c_double), ("mu_s", C.c_double),
        ("c_tol", C.c_double), ("mass_spacing", C.c_double),
    ]


class LbmParticle(C.Structure):
    _fields_ = [
        ("n_cp", C.c_int32), ("fixed", C.c_int32),
        ("cp", (C.c_double * 3) * MAX_CP), ("K", C.c_double * MAX_CP),
        ("Rs", C.c_double), ("density", C.c_double), ("mass", C.c_double),
        ("inertia", C.c_double * 9),
        ("x", C.c_double * 3), ("q", C.c_double * 4), ("v", C.c_double * 3), ("w", C.c_double * 3),
    ]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# Exported C-ABI functions and their ctypes signatures (the header declares
# exactly these).
_SIGS = {
    "lbm_workspace_size": (C.c_int, [C.POINTER(LbmConfig), C.POINTER(C.c_size_t)]),
    "lbm_init": (C.c_int, [C.POINTER(LbmConfig), C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_set_particles": (C.c_int, [C.c_void_p, C.POINTER(LbmParticle), C.c_int]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_get_forces": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(LbmParticle)]),
    "lbm_get_contact_forces": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_get_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_set_populations": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_get_populations": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_check": (C.c_int, [C.c_void_p]),
    "lbm_get_counters": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]),
    "lbm_kernels_per_step": (C.c_int, [C.c_void_p]),
    "lbm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_profile_mask": (C.c_int, [C.c_void_p, C.c_uint, C.c_int]),
    "lbm_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "lbm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lbm_set_plain_speculation": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_batch_workspace_size": (C.c_int, [C.POINTER(LbmConfig), C.c_int, C.POINTER(C.c_size_t)]),
    "lbm_batch_init": (C.c_int, [C.POINTER(LbmConfig), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    "lbm_batch_set_particles": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(LbmParticle), C.c_int]),
    "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_batch_get_forces": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_batch_get_all_forces": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_batch_get_populations": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lbm_batch_set_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lbm_batch_tune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_double)]),
    "lbm_batch_steps": (C.c_int64, [C.c_void_p]),
    "lbm_batch_destroy": (C.c_int, [C.c_void_p]),
    "lbm_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_adj_workspace_size": (C.c_int, [C.POINTER(LbmConfig), C.POINTER(LbmParticle), C.c_int, C.c_int,
                                         C.POINTER(C.c_size_t)]),
    "lbm_adj_init": (C.c_int, [C.POINTER(LbmConfig), C.POINTER(LbmParticle), C.c_int, C.c_int, C.c_void_p,
                               C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_adj_forward": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_adj_backward": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lbm_adj_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lbm_adj_destroy": (C.c_int, [C.c_void_p]),
    "lbm_adj_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_flags_noalloc": (C.c_int, [C.POINTER(LbmConfig), C.POINTER(LbmParticle), C.c_int, C.c_void_p, C.c_void_p]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
}


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load liblbmmb.so (built by __graft_entry__.build()); raises when absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() first")
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def make_config(nx: int, ny: int, nz: int, *, lattice: int = 19, storage: str | int = "f32",
                periodic=(0, 0, 0), n_sub: int = 0, vibb: int = 1, missing_force: int = 1,
                max_particles: int = 1, tau: float = 0.8, rho0: float = 1.0, c0: float = 1.0,
                u0=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0),
                kn: float = 0.0, eta_n: float = 0.0, kt: float = 0.0, eta_t: float = 0.0, mu_s: float = 0.0,
                c_tol: float = 1e-6, mass_spacing: float = 0.5, dem_mode: int = 0, q_exact: int = 0) -> LbmConfig:
    c = LbmConfig()
    c.nx, c.ny, c.nz = nx, ny, nz
    c.lattice = lattice
    c.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    for a in range(3):
        c.periodic[a] = int(periodic[a])
        c.u0[a], c.force[a], c.gravity[a] = u0[a], force[a], gravity[a]
    c.n_sub, c.vibb, c.missing_force, c.max_particles = n_sub, vibb, missing_force, max_particles
    c.tau, c.rho0, c.c0 = tau, rho0, c0
    c.kn, c.eta_n, c.kt, c.eta_t, c.mu_s, c.c_tol = kn, eta_n, kt, eta_t, mu_s, c_tol
    c.mass_spacing = mass_spacing
    c.dem_mode = int(dem_mode)
    c.q_exact = int(q_exact)
    return c


def make_particle(cp: Sequence[Sequence[float]], K: Sequence[float], x, *, q=(1, 0, 0, 0), v=(0, 0, 0),
                  w=(0, 0, 0), Rs=0.0, density=1.0, mass=0.0, inertia=None, fixed=0) -> LbmParticle:
    p = LbmParticle()
    cp = np.asarray(cp, dtype=np.float64).reshape(-1, 3)
    if not 1 <= len(cp) <= MAX_CP or len(K) != len(cp):
        raise ValueError("1..16 control points with one weight each")
    p.n_cp, p.fixed = len(cp), int(fixed)
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


def particle_dict(p: LbmParticle) -> dict:
    n = p.n_cp
    return dict(n_cp=n, fixed=p.fixed, cp=np.array([[p.cp[k][a] for a in range(3)] for k in range(n)]),
                K=np.array([p.K[k] for k in range(n)]), Rs=p.Rs, density=p.density, mass=p.mass,
                inertia=np.array(list(p.inertia)).reshape(3, 3), x=np.array(list(p.x)), q=np.array(list(p.q)),
                v=np.array(list(p.v)), w=np.array(list(p.w)))


class Lattice:
    """One lattice with its flags and particles, stepped on the GPU."""

    def __init__(self, nx: int, ny: int, nz: int, *, device: str = "cuda", stream=None, **kw):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.L = load_library()
        self.torch = torch
        self.cfg = make_config(nx, ny, nz, **kw)
        self.Q = self.cfg.lattice
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        size = C.c_size_t()
        self._ok(self.L.lbm_workspace_size(C.byref(self.cfg), C.byref(size)), None)
        self.ws_bytes = size.value
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.L.lbm_init(C.byref(self.cfg), C.c_void_p(self.ws.data_ptr()), self.ws_bytes,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h))
        self._ok(rc, None)
        self.h = h
        self.np = 0

    def _ok(self, rc: int, h) -> None:
        if rc != 0:
            msg = self.L.lbm_last_error(h).decode()
            raise LbmError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # particles -------------------------------------------------------------
    def set_particles(self, particles: Iterable[LbmParticle]) -> None:
        plist = list(particles)
        arr = (LbmParticle * max(1, len(plist)))(*plist)
        self._ok(self.L.lbm_set_particles(self.h, arr, len(plist)), self.h)
        self.np = len(plist)

    def forces(self):
        n = max(1, self.np)
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        self._ok(self.L.lbm_get_forces(self.h, F.ctypes.data_as(C.POINTER(C.c_double)),
                                       T.ctypes.data_as(C.POINTER(C.c_double)), None), self.h)
        return F[: self.np], T[: self.np]

    def contact_forces(self):
        n = max(1, self.np)
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        self._ok(self.L.lbm_get_contact_forces(self.h, F.ctypes.data_as(C.POINTER(C.c_double)),
                                               T.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return F[: self.np], T[: self.np]

    def particles(self) -> list[dict]:
        arr = (LbmParticle * max(1, self.np))()
        self._ok(self.L.lbm_get_forces(self.h, None, None, arr), self.h)
        return [particle_dict(arr[j]) for j in range(self.np)]

    # stepping ----------------------------------------------------------------
    def step(self, n: int = 1) -> None:
        self._ok(self.L.lbm_step(self.h, int(n)), self.h)

    def set_schedule(self, plain_ctas_per_sm: int, chain_ctas_per_sm: int) -> None:
        self._ok(self.L.lbm_set_schedule(self.h, int(plain_ctas_per_sm), int(chain_ctas_per_sm)), self.h)

    def set_plain_speculation(self, mode: int) -> None:
        """1: the plain sweep pulls before reading its near-set entry, 0: after,
        -1: chosen from the particles' extent (lbm_set_plain_speculation)."""
        self._ok(self.L.lbm_set_plain_speculation(self.h, int(mode)), self.h)

    def kernels_per_step(self) -> int:
        return self.L.lbm_kernels_per_step(self.h)

    # state -------------------------------------------------------------------
    def fields(self):
        t = self.torch
        rho = t.empty(self.shape, dtype=t.float64, device=self.device)
        u = t.empty((3,) + self.shape, dtype=t.float64, device=self.device)
        fl = t.empty(self.shape, dtype=t.int16, device=self.device)
        self._ok(self.L.lbm_get_fields(self.h, C.c_void_p(rho.data_ptr()), C.c_void_p(u.data_ptr()),
                                       C.c_void_p(fl.data_ptr())), self.h)
        return rho, u, fl.view(t.uint16) if hasattr(t, "uint16") else fl

    def flags(self):
        """Node flags as int32 on the device: 0 fluid, j+1 solid of particle j."""
        t = self.torch
        fl = t.empty(self.shape, dtype=t.int16, device=self.device)
        self._ok(self.L.lbm_get_fields(self.h, None, None, C.c_void_p(fl.data_ptr())), self.h)
        return fl.to(t.int32) & 0xFFFF

    def populations(self):
        t = self.torch
        f = t.empty((self.Q,) + self.shape, dtype=t.float64, device=self.device)
        self._ok(self.L.lbm_get_populations(self.h, C.c_void_p(f.data_ptr())), self.h)
        return f

    def set_populations(self, f) -> None:
        t = self.torch
        f = t.as_tensor(f, dtype=t.float64, device=self.device).contiguous()
        if tuple(f.shape) != (self.Q,) + self.shape:
            raise ValueError(f"populations must have shape {(self.Q,) + self.shape}")
        self._ok(self.L.lbm_set_populations(self.h, C.c_void_p(f.data_ptr())), self.h)

    def check(self) -> None:
        self._ok(self.L.lbm_check(self.h), self.h)

    KERNELS = ("k_bin", "k_flags", "k_sweep_plain", "k_sweep_near", "k_force_reduce", "k_dem", "k_sweep_near_plain")

    def profile(self, enable: bool = True, kernels=None, every: int = 1) -> None:
        """Record event pairs around every kernel (enable), or only around the
        named ones (kernels: names from KERNELS), on every every-th launch."""
        if enable and kernels is not None:
            mask = 0
            for name in kernels:
                mask |= 1 << self.KERNELS.index(name)
            self._ok(self.L.lbm_profile_mask(self.h, mask, int(every)), self.h)
        else:
            self._ok(self.L.lbm_profile(self.h, int(enable)), self.h)

    def profile_read(self) -> dict:
        """{kernel: (total_ms, launches)} recorded since profile(True)."""
        out = {}
        for k, name in enumerate(self.KERNELS):
            ms, n = C.c_double(), C.c_int64()
            self._ok(self.L.lbm_profile_read(self.h, k, C.byref(ms), C.byref(n)), self.h)
            out[name] = (ms.value, n.value)
        return out

    def counters(self) -> dict:
        st, nr, nl, nb = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        self._ok(self.L.lbm_get_counters(self.h, C.byref(st), C.byref(nr), C.byref(nl), C.byref(nb)), self.h)
        return dict(step=st.value, nrefill=nr.value, nlinks=nl.value, near_bricks=nb.value)


class Batch:
    """Independent lattices stepped together (lbm_batch_*): one launch per
    phase for all cases, the steps of a call run as a captured CUDA graph.
    cases: list of make_config keyword dicts, each with nx, ny, nz."""

    def __init__(self, cases: list, *, device: str = "cuda", stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.L = load_library()
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = len(cases)
        self.cfgs = (LbmConfig * n)()
        self.shapes = []
        for c, kw in enumerate(cases):
            kw = dict(kw)
            nx, ny, nz = kw.pop("nx"), kw.pop("ny"), kw.pop("nz")
            self.cfgs[c] = make_config(nx, ny, nz, **kw)
            self.shapes.append((nz, ny, nx))
        self.n = n
        self.Q = self.cfgs[0].lattice
        size = C.c_size_t()
        self._ok(self.L.lbm_batch_workspace_size(self.cfgs, n, C.byref(size)), None)
        self.ws_bytes = size.value
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.L.lbm_batch_init(self.cfgs, n, C.c_void_p(self.ws.data_ptr()), self.ws_bytes,
                                       C.c_void_p(self.stream.cuda_stream), C.byref(h))
        self._ok(rc, None)
        self.h = h
        self.np = [0] * n

    def _ok(self, rc: int, h) -> None:
        if rc != 0:
            raise LbmError(rc, self.L.lbm_batch_last_error(h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, c: int, particles: Iterable[LbmParticle]) -> None:
        plist = list(particles)
        arr = (LbmParticle * max(1, len(plist)))(*plist)
        self._ok(self.L.lbm_batch_set_particles(self.h, c, arr, len(plist)), self.h)
        self.np[c] = len(plist)

    def step(self, n: int = 1) -> None:
        self._ok(self.L.lbm_batch_step(self.h, int(n)), self.h)

    @property
    def steps(self) -> int:
        return int(self.L.lbm_batch_steps(self.h))

    def forces(self, c: int):
        n = max(1, self.np[c])
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        self._ok(self.L.lbm_batch_get_forces(self.h, c, F.ctypes.data_as(C.POINTER(C.c_double)),
                                             T.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return F[: self.np[c]], T[: self.np[c]]

    def all_forces(self):
        """Force and torque of every case's particles, cases in order: two
        (sum of particle counts, 3) arrays, read with one wait."""
        n = max(1, sum(self.np))
        F = np.zeros((n, 3))
        T = np.zeros((n, 3))
        self._ok(self.L.lbm_batch_get_all_forces(self.h, F.ctypes.data_as(C.POINTER(C.c_double)),
                                                 T.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return F[: sum(self.np)], T[: sum(self.np)]

    def populations(self, c: int):
        t = self.torch
        f = t.empty((self.Q,) + self.shapes[c], dtype=t.float64, device=self.device)
        self._ok(self.L.lbm_batch_get_populations(self.h, c, C.c_void_p(f.data_ptr())), self.h)
        return f

    def set_schedule(self, chain_ctas_per_case: int, plain_blocks_per_cta: int) -> None:
        self._ok(self.L.lbm_batch_set_schedule(self.h, int(chain_ctas_per_case), int(plain_blocks_per_cta)), self.h)

    def tune(self, trial_steps: int = 5):
        g, k, ms = C.c_int(), C.c_int(), C.c_double()
        self._ok(self.L.lbm_batch_tune(self.h, int(trial_steps), C.byref(g), C.byref(k), C.byref(ms)), self.h)
        return g.value, k.value, ms.value
