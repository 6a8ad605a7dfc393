"""FP64 oracle of the learned closure trained through the pressure projection.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper motivates machine-learned subgrid/wall closures developed on top of
the solver (Sec. 1) and performs the projection step of Eqs. (12)-(13):
u = u* - grad(phi) with L phi = div u* (the factor gamma*dt cancels).  Here:

  P(u)          = u - grad(S(div u))       S = Poisson solve of ``solve``
  N_theta(u)_c  = sum_t theta[c, t] u_c(x + o_t)   (27-tap stencil per component)
  prediction    = P(u + N_theta(u))
  target        = P(G(u)),  G(u)_c = u_c + kappa*Lap27(u_c) + beta*tanh(u_c)
  loss          = mean over all velocity points of (prediction - target)^2

Stencil boundary handling: x and y wrap (periodic); z reads zero outside the
component's planes (nz planes for u, v; nz+1 faces for w); the wall faces of w
(0 and nz) are held at zero on output.
"""
from __future__ import annotations

import numpy as np

from .cales_oracle import Grid, divergence, divergence_T, gradient, gradient_T, solve, solve_T

__all__ = ["OFFSETS", "stencil_apply", "stencil_weight_grad", "hidden_operator",
           "project_velocity", "project_velocity_T", "closure_loss", "closure_loss_grad",
           "HIDDEN_KAPPA", "HIDDEN_BETA"]

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
HIDDEN_KAPPA = 0.5
HIDDEN_BETA = 0.1


def _shift(a: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """b[k,j,i] = a[k+dz, j+dy, i+dx]; periodic in j, i; zero outside in k."""
    b = np.roll(a, (-dy, -dx), axis=(1, 2))
    if dz == 0:
        return b
    out = np.zeros_like(b)
    if dz > 0:
        out[:-dz] = b[dz:]
    else:
        out[-dz:] = b[:dz]
    return out


def _mask_walls(comp: int, a: np.ndarray) -> np.ndarray:
    if comp == 2:
        a = a.copy()
        a[0] = 0.0
        a[-1] = 0.0
    return a


def stencil_apply(theta: np.ndarray, vel):
    """N_theta(u) for the three components; theta is (3, 27)."""
    out = []
    for c, a in enumerate(vel):
        acc = np.zeros_like(a)
        for t, (dz, dy, dx) in enumerate(OFFSETS):
            acc += theta[c, t] * _shift(a, dz, dy, dx)
        out.append(_mask_walls(c, acc))
    return out


def stencil_weight_grad(gout, vel) -> np.ndarray:
    """d/dtheta of sum_c <gout_c, N_theta(u)_c> (outputs at w walls are fixed)."""
    g = np.zeros((3, 27))
    for c, (go, a) in enumerate(zip(gout, vel)):
        go = _mask_walls(c, go)
        for t, (dz, dy, dx) in enumerate(OFFSETS):
            g[c, t] = float((go * _shift(a, dz, dy, dx)).sum())
    return g


def hidden_operator(vel, kappa: float = HIDDEN_KAPPA, beta: float = HIDDEN_BETA):
    """Ground-truth map G that the closure has to learn (a 27-point index
    Laplacian plus a small non-linearity the linear stencil cannot represent)."""
    theta = np.full((3, 27), kappa / 26.0)
    theta[:, 13] = -kappa
    lap = stencil_apply(theta, vel)
    return [_mask_walls(c, a + l + beta * np.tanh(a)) for c, (a, l) in enumerate(zip(vel, lap))]


def project_velocity(vel, g: Grid):
    """P(u) = u - grad S(div u)."""
    phi = solve(divergence(*vel, g), g)
    gx, gy, gz = gradient(phi, g)
    return [vel[0] - gx, vel[1] - gy, vel[2] - gz]


def project_velocity_T(r, g: Grid):
    """P^T r = r - div^T S^T grad^T r."""
    s = solve_T(gradient_T(*r, g), g)
    ux, vy, wz = divergence_T(s, g)
    return [r[0] - ux, r[1] - vy, r[2] - wz]


def _npts(vel) -> int:
    return sum(a.size for a in vel)


def closure_loss(theta, vel, target, g: Grid) -> float:
    pred = project_velocity([a + n for a, n in zip(vel, stencil_apply(theta, vel))], g)
    return float(sum(((p - t) ** 2).sum() for p, t in zip(pred, target)) / _npts(vel))


def closure_loss_grad(theta, vel, target, g: Grid):
    """(loss, dloss/dtheta) by the transposed chain: stencil^T P^T (2 e / N)."""
    pred = project_velocity([a + n for a, n in zip(vel, stencil_apply(theta, vel))], g)
    npts = _npts(vel)
    err = [p - t for p, t in zip(pred, target)]
    loss = float(sum((e ** 2).sum() for e in err) / npts)
    gpred = [2.0 * e / npts for e in err]
    gin = project_velocity_T(gpred, g)
    return loss, stencil_weight_grad(gin, vel)
