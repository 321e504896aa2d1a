"""Differentiable rollout: the final velocity after T steps as a function of
the initial velocity and the viscosity, with gradients from the library's
hand-written discrete adjoint and sqrt(T) checkpointing (recomputation of
each segment from its checkpoint).  All arithmetic runs in the CUDA library;
this module only moves tensors in and out of the grid.
"""
from __future__ import annotations

import math

from .grid import Grid, U, V, W, P, LU, LV, LW, LP, mask


class Rollout:
    """A periodic FP32 block (ghost width 2) stepped nsteps times with dt.

    rollout(u0, v0, w0, nu) -> (uT, vT, wT); u0.. are (nz, ny, nx) float32
    CUDA tensors, nu a 0-d tensor.  Gradients flow to u0, v0, w0 and nu.
    p starts at zero (the Jacobi warm start).  form: the advection term,
    'advective' or 'flux'."""

    def __init__(self, dims, h, nsteps, dt, jacobi_iters=50, omega=1.0, seg=None, stream=None,
                 form="advective"):
        import torch
        self.torch = torch
        self.grid = Grid(dims, ghost=2, h=h, dtype="f32", stream=stream)
        self.grid.set_advection(form)
        self.nsteps, self.dt = int(nsteps), float(dt)
        self.iters, self.omega = int(jacobi_iters), float(omega)
        self.seg = int(seg) if seg else max(1, int(math.ceil(math.sqrt(self.nsteps))))
        self.nbytes = self.grid.rollout_bytes(self.nsteps, self.seg)
        with torch.cuda.stream(self.grid.stream):
            self.store = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        self.store_ptr = self.store.data_ptr() + ((-self.store.data_ptr()) % 256)

    def __call__(self, u0, v0, w0, nu):
        return _RolloutFn.apply(u0, v0, w0, nu, self)

    def forward_only(self, u0, v0, w0, nu):
        """The same rollout without recording a graph for autograd."""
        with self.torch.no_grad():
            return _RolloutFn.run_forward(self, u0, v0, w0, float(nu))


class _RolloutFn:
    pass


def _make_fn():
    import torch

    class RolloutFn(torch.autograd.Function):
        @staticmethod
        def run_forward(ro, u0, v0, w0, nu):
            g = ro.grid
            g.set_params(nu, ro.iters, ro.omega, 2)
            with torch.cuda.stream(g.stream):
                for a, x in ((U, u0), (V, v0), (W, w0)):
                    g.interior(a).copy_(x)
                g.interior(P).zero_()
            g.ghost_fill(mask(U, V, W, P))
            g.rollout_forward(ro.dt, ro.nsteps, ro.seg, ro.store_ptr, ro.nbytes)
            with torch.cuda.stream(g.stream):
                return tuple(g.interior(a).clone() for a in (U, V, W))

        @staticmethod
        def forward(ctx, u0, v0, w0, nu, ro):
            ctx.ro = ro
            ctx.nu_meta = (nu.dtype, nu.device)
            return RolloutFn.run_forward(ro, u0, v0, w0, float(nu))

        @staticmethod
        def backward(ctx, gu, gv, gw):
            ro = ctx.ro
            g = ro.grid
            with torch.cuda.stream(g.stream):
                for a, x in ((LU, gu), (LV, gv), (LW, gw)):
                    if x is None:
                        g.interior(a).zero_()
                    else:
                        g.interior(a).copy_(x)
                g.interior(LP).zero_()
            dnu = g.rollout_backward(ro.dt, ro.nsteps, ro.seg, ro.store_ptr, ro.nbytes)
            with torch.cuda.stream(g.stream):
                grads = tuple(g.interior(a).clone() for a in (LU, LV, LW))
            dtype, device = ctx.nu_meta
            return grads + (torch.tensor(dnu, dtype=dtype, device=device), None)

    return RolloutFn


_RolloutFn = _make_fn()
