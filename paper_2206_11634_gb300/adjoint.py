"""Drag gradient with respect to a fixed metaball's shape (the C ABI of
include/lbm_adjoint.h): the library's hand-written discrete adjoint of the
sweep, the interpolated bounce-back and the momentum exchange, with the node
flags frozen, wrapped as a torch.autograd.Function.

    drag = AdjointDrag(nx=96, ny=96, nz=96, tau=0.55, u0=(U, 0, 0), force=(Fx, 0, 0),
                       particle=make_particle(...), T=500, W=100)
    cp = torch.tensor(world_control_points, dtype=torch.float64, requires_grad=True)
    K = torch.tensor(weights, dtype=torch.float64, requires_grad=True)
    J = drag(cp, K)          # mean F_x over the last W of T steps
    J.backward()             # cp.grad, K.grad

Marshalling only: the forward run, the adjoint and the chain rule to the
control points all run on the GPU.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .lbm import LbmConfig, LbmError, LbmParticle, load_library, make_config


class AdjointDrag:
    def __init__(self, nx: int, ny: int, nz: int, *, particle: LbmParticle, T: int, W: int, device: str = "cuda",
                 stream=None, **kw):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.L = load_library()
        self.torch = torch
        kw.setdefault("periodic", (1, 1, 1))
        self.cfg: LbmConfig = make_config(nx, ny, nz, **kw)
        self.particle = particle
        self.ncp = int(particle.n_cp)
        self.T, self.W = int(T), int(W)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        size = C.c_size_t()
        self._ok(self.L.lbm_adj_workspace_size(C.byref(self.cfg), C.byref(particle), self.T, self.W, C.byref(size)),
                 None)
        self.ws = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.L.lbm_adj_init(C.byref(self.cfg), C.byref(particle), self.T, self.W,
                                     C.c_void_p(self.ws.data_ptr()), size.value, C.c_void_p(self.stream.cuda_stream),
                                     C.byref(h))
        self._ok(rc, None)
        self.h = h

    def _ok(self, rc: int, h) -> None:
        if rc != 0:
            raise LbmError(rc, self.L.lbm_adj_last_error(h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_adj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        n, k = C.c_int(), C.c_int()
        self._ok(self.L.lbm_adj_info(self.h, C.byref(n), C.byref(k)), self.h)
        return dict(nlinks=n.value, checkpoint_every=k.value)

    def forward_np(self, cp_world, K) -> float:
        cp = np.ascontiguousarray(np.asarray(cp_world, dtype=np.float64).reshape(self.ncp, 3))
        Kv = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(self.ncp))
        J = C.c_double()
        self._ok(self.L.lbm_adj_forward(self.h, cp.ctypes.data_as(C.POINTER(C.c_double)),
                                        Kv.ctypes.data_as(C.POINTER(C.c_double)), C.byref(J)), self.h)
        return J.value

    def backward_np(self):
        dcp = np.zeros((self.ncp, 3))
        dK = np.zeros(self.ncp)
        self._ok(self.L.lbm_adj_backward(self.h, dcp.ctypes.data_as(C.POINTER(C.c_double)),
                                         dK.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return dcp, dK

    def __call__(self, cp_world, K):
        return _MetaballDrag.apply(cp_world, K, self)


def _function():
    import torch

    class MetaballDrag(torch.autograd.Function):
        """J(control points, weights) = mean drag over the window; backward
        runs the library's adjoint of that forward run."""

        @staticmethod
        def forward(ctx, cp_world, K, engine):
            J = engine.forward_np(cp_world.detach().cpu().numpy(), K.detach().cpu().numpy())
            ctx.engine = engine
            ctx.dev = (cp_world.device, cp_world.dtype, K.device, K.dtype)
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            dcp, dK = ctx.engine.backward_np()
            d0, t0, d1, t1 = ctx.dev
            g = float(gJ)
            return (torch.as_tensor(dcp * g, dtype=t0, device=d0), torch.as_tensor(dK * g, dtype=t1, device=d1),
                    None)

    return MetaballDrag


class _Lazy:
    fn = None

    @classmethod
    def apply(cls, *a):
        if cls.fn is None:
            cls.fn = _function()
        return cls.fn.apply(*a)


_MetaballDrag = _Lazy
