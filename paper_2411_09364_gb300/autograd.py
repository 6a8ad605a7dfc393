"""Differentiable solves and the differentiable pressure projection.

``poisson_solve(f, plan)`` and ``helmholtz_solve(f, plan, alpha)`` are
``torch.autograd.Function``s whose backward is the library's adjoint solve
(transposed tridiagonal systems around the same transforms).  ``project``
applies P(u) = u - grad S(div u), the pressure projection of the fractional
step (Sec. 2.2, Eqs. 12-13, gamma*dt folded into phi); its backward is
P^T r = r - div^T S^T grad^T r, every operator a library kernel.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N
from .solver import Plan, _stream


def _vp(t):
    return C.c_void_p(t.data_ptr() if t is not None else 0)


class _PoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, plan):
        ctx.plan = plan
        return plan.poisson(f.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.poisson_adjoint(g.contiguous()), None


class _HelmholtzSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, plan, alpha):
        ctx.plan, ctx.alpha = plan, alpha
        return plan.helmholtz(alpha, f.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.helmholtz_adjoint(ctx.alpha, g.contiguous()), None, None


def poisson_solve(f: torch.Tensor, plan: Plan) -> torch.Tensor:
    """p = S f (Eq. 12), differentiable in f."""
    return _PoissonSolve.apply(f, plan)


def helmholtz_solve(f: torch.Tensor, plan: Plan, alpha: float) -> torch.Tensor:
    """u = (I - alpha L)^-1 f (Eq. 18), differentiable in f."""
    return _HelmholtzSolve.apply(f, plan, alpha)


# --------------------------------------------------------------------------
# staggered operators (plans periodic in x, y with wall z sides)
# --------------------------------------------------------------------------
def _shapes(plan):
    return (plan.nz, plan.ny, plan.nx), (plan.nz + 1, plan.ny, plan.nx)


def divergence(plan: Plan, u, v, w, out=None):
    c, _ = _shapes(plan)
    d = torch.empty(c, dtype=u.dtype, device=u.device) if out is None else out
    N.check(N.lib().cales_divergence(plan.handle, _vp(u), _vp(v), _vp(w), _vp(d), _stream(None)), "cales_divergence")
    return d


def gradient(plan: Plan, phi, sub=None):
    """grad phi, or (u, v, w) - grad phi when ``sub`` = (u, v, w)."""
    c, f = _shapes(plan)
    gx = torch.empty(c, dtype=phi.dtype, device=phi.device)
    gy = torch.empty(c, dtype=phi.dtype, device=phi.device)
    gz = torch.empty(f, dtype=phi.dtype, device=phi.device)
    uin, vin, win = sub if sub is not None else (None, None, None)
    N.check(N.lib().cales_gradient(plan.handle, _vp(phi), _vp(uin), _vp(vin), _vp(win), _vp(gx), _vp(gy), _vp(gz),
                                   _stream(None)), "cales_gradient")
    return gx, gy, gz


def divergence_T(plan: Plan, d, sub=None):
    """div^T d, or (u, v, w) - div^T d when ``sub`` = (u, v, w)."""
    c, f = _shapes(plan)
    u = torch.empty(c, dtype=d.dtype, device=d.device)
    v = torch.empty(c, dtype=d.dtype, device=d.device)
    w = torch.empty(f, dtype=d.dtype, device=d.device)
    uin, vin, win = sub if sub is not None else (None, None, None)
    N.check(N.lib().cales_divergence_adjoint(plan.handle, _vp(d), _vp(uin), _vp(vin), _vp(win), _vp(u), _vp(v),
                                             _vp(w), _stream(None)), "cales_divergence_adjoint")
    return u, v, w


def gradient_T(plan: Plan, gx, gy, gz):
    c, _ = _shapes(plan)
    phi = torch.empty(c, dtype=gx.dtype, device=gx.device)
    N.check(N.lib().cales_gradient_adjoint(plan.handle, _vp(gx), _vp(gy), _vp(gz), _vp(phi), _stream(None)),
            "cales_gradient_adjoint")
    return phi


def project_forward(plan: Plan, u, v, w):
    phi = plan.poisson(divergence(plan, u, v, w))
    return gradient(plan, phi, sub=(u, v, w))


def project_backward(plan: Plan, gu, gv, gw):
    s = plan.poisson_adjoint(gradient_T(plan, gu, gv, gw))
    return divergence_T(plan, s, sub=(gu, gv, gw))


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, v, w, plan):
        ctx.plan = plan
        return project_forward(plan, u.contiguous(), v.contiguous(), w.contiguous())

    @staticmethod
    def backward(ctx, gu, gv, gw):
        return (*project_backward(ctx.plan, gu.contiguous(), gv.contiguous(), gw.contiguous()), None)


def project(u, v, w, plan: Plan):
    """P(u) = u - grad S(div u), differentiable in (u, v, w)."""
    return _Project.apply(u, v, w, plan)
