"""Learned closure trained through the pressure projection.

The paper develops its solver as a platform for machine-learned subgrid and
wall closures (Sec. 1).  Here a closure N_theta (a 27-tap stencil per velocity
component, FP32) corrects the provisional velocity before the projection of
the fractional step (Sec. 2.2, Eqs. 12-13):

    prediction = P(u + N_theta(u)),   P(u) = u - grad S(div u)

and is fitted to targets P(G(u)) of a hidden operator G.  Forward, loss,
backward through P^T (adjoint solve), weight gradient and the Adam update all
run in the library's CUDA kernels; torch provides memory only.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from .autograd import _vp, project_backward, project_forward
from .solver import Plan, _stream

HIDDEN_KAPPA = 0.5
HIDDEN_BETA = 0.1


def _ptrs(ts):
    return (C.c_void_p * 3)(*[t.data_ptr() if t is not None else 0 for t in ts])


def hidden_theta(device, kappa: float = HIDDEN_KAPPA) -> torch.Tensor:
    """Taps of the 27-point index Laplacian kappa * (sum of neighbours - 26 u) / 26."""
    th = torch.full((3, 27), kappa / 26.0, dtype=torch.float32)
    th[:, 13] = -kappa
    return th.to(device)


class StencilClosure:
    """27-tap stencil closure with its Adam state, bound to an FP32 channel plan."""

    def __init__(self, plan: Plan, lr: float = 2e-2, betas=(0.9, 0.999), eps: float = 1e-8):
        if plan.dtype != torch.float32:
            raise ValueError("the closure runs on an FP32 plan")
        self.plan = plan
        dev = torch.device("cuda", torch.cuda.current_device())
        self.theta = torch.zeros((3, 27), dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.gacc = torch.zeros((3, 27), dtype=torch.float64, device=dev)
        self.lacc = torch.zeros(1, dtype=torch.float64, device=dev)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.t = 0

    # -- operators ----------------------------------------------------------
    def stencil(self, vel, theta=None, a: float = 1.0, beta: float = 0.0):
        th = self.theta if theta is None else theta
        out = [torch.empty_like(x) for x in vel]
        N.check(N.lib().cales_stencil27(self.plan.handle, _vp(th), C.c_float(a), C.c_float(beta), _ptrs(vel),
                                        _ptrs(out), _stream(None)), "cales_stencil27")
        return out

    def target(self, vel, kappa: float = HIDDEN_KAPPA, beta: float = HIDDEN_BETA):
        """P(G(u)) with G(u) = u + kappa Lap27(u) + beta tanh(u)."""
        g = self.stencil(vel, hidden_theta(vel[0].device, kappa), 1.0, beta)
        return project_forward(self.plan, *g)

    def _zero(self, t):
        N.check(N.lib().cales_zero(_vp(t), C.c_ulong(t.numel() * t.element_size()), _stream(None)), "cales_zero")

    def loss(self, vel, target, theta=None, with_grad: bool = False):
        """Mean squared error of P(u + N_theta u) against the target; optionally
        leaves d loss / d theta (FP64) in ``self.gacc``."""
        x = self.stencil(vel, theta, 1.0, 0.0)
        pred = project_forward(self.plan, *x)
        npts = sum(p.numel() for p in pred)
        grads = [torch.empty_like(p) for p in pred] if with_grad else None
        self._zero(self.lacc)
        n = (C.c_long * 3)(*[p.numel() for p in pred])
        N.check(N.lib().cales_sq_error(_ptrs(pred), _ptrs(target), _ptrs(grads) if grads else None, n,
                                       C.c_float(2.0 / npts), _vp(self.lacc), _stream(None)), "cales_sq_error")
        if with_grad:
            gin = project_backward(self.plan, *grads)
            self._zero(self.gacc)
            N.check(N.lib().cales_stencil27_weight_grad(self.plan.handle, _ptrs(gin), _ptrs(vel), _vp(self.gacc),
                                                        _stream(None)), "cales_stencil27_weight_grad")
        return float(self.lacc.item()) / npts

    def step(self, vel, target):
        """One Adam step on one sample; returns the loss before the update."""
        loss = self.loss(vel, target, with_grad=True)
        self.t += 1
        N.check(N.lib().cales_adam_step(_vp(self.theta), _vp(self.gacc), _vp(self.m), _vp(self.v), 81,
                                        C.c_float(self.lr), C.c_float(self.betas[0]), C.c_float(self.betas[1]),
                                        C.c_float(self.eps), self.t, C.c_float(1.0), _stream(None)),
                "cales_adam_step")
        return loss
