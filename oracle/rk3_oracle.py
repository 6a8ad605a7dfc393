"""FP64 oracle of the explicit low-storage RK3 pressure-correction substep.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2, Eqs. 11-14 with the explicit viscous term (Algorithm 1):
    u*        = u^k + dt [alpha (H^k + nu L u^k) + beta (H^{k-1} + nu L u^{k-1}) - gamma grad p^{k-1/2}]
    L phi     = div u* / (gamma dt)
    u^{k+1}   = u* - gamma dt grad phi
    p^{k+1/2} = p^{k-1/2} + phi
followed by nu_t^{k+1} from u^{k+1} (Eq. 4).  alpha, beta, gamma are the
Wray coefficients printed below Eq. 14.  The paper leaves open, read here as:

T1  signs of H_i (Eq. 15) from the momentum equation (Eq. 2) and the
    Boussinesq closure (Eq. 3): H_i = -d(u_i u_j)/dx_j + d(2 nu_t S_ij)/dx_j;
    the right-hand side carried between substeps is R = H + nu L u;
T2  advection in divergence form on the staggered grid, every interpolated
    velocity the arithmetic mean of its two neighbours (also in stretched z);
T3  channel: x, y periodic, no-slip walls in z (u, v ghosts minus the first
    interior value at the distances dzc[0], dzc[nz]; w = 0 on the wall faces);
    strain rates as the eddy-viscosity oracle forms them on cell edges;
T4  nu_t on an edge is the mean of the four cell centres around it; beyond a
    wall the ghost centre repeats the first interior value.

Layout as the rest of the oracle: u [nz][ny][nx] on x-faces i+1/2, v on
y-faces j+1/2, w [nz+1][ny][nx] on z-faces, p, nu_t at cell centres.
"""
from __future__ import annotations

import numpy as np

from .cales_oracle import Grid, divergence, gradient, solve
from .sgs_oracle import eddy_viscosity

__all__ = ["RK3_ALPHA", "RK3_BETA", "RK3_GAMMA", "advection", "viscous", "sgs_divergence", "momentum_rhs",
           "rk3_substep"]

RK3_ALPHA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_BETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)
RK3_GAMMA = tuple(a + b for a, b in zip(RK3_ALPHA, RK3_BETA))


def _x(a, s):
    """a at i + s (periodic x)."""
    return np.roll(a, -s, axis=2)


def _y(a, s):
    """a at j + s (periodic y)."""
    return np.roll(a, -s, axis=1)


def _ghost(c, sign):
    """Cell-centred (in z) field with one ghost plane on either side: rows
    -1 and nz hold sign * (first / last interior row).  Index k + 1."""
    return np.concatenate([sign * c[:1], c, sign * c[-1:]], axis=0)


def _col(a):
    return np.asarray(a).reshape(-1, 1, 1)


def advection(u, v, w, g: Grid):
    """Divergence-form advection d(u_i u_j)/dx_j at the u, v, w points (T2);
    the w rows 0 and nz (walls) are zero."""
    ue, ve = _ghost(u, -1.0), _ghost(v, -1.0)
    # u-momentum: centre fluxes in x, (i+1/2, j+1/2) edges in y, (i+1/2, face k) edges in z
    fxx = (0.5 * (_x(u, -1) + u)) ** 2                        # centre i
    fxy = 0.5 * (u + _y(u, 1)) * 0.5 * (v + _x(v, 1))         # edge (i+1/2, j+1/2)
    fxz = 0.5 * (ue[:-1] + ue[1:]) * 0.5 * (w + _x(w, 1))     # edge (i+1/2, face k), k = 0..nz
    fyy = (0.5 * (_y(v, -1) + v)) ** 2                        # centre j
    fyz = 0.5 * (ve[:-1] + ve[1:]) * 0.5 * (w + _y(w, 1))     # edge (j+1/2, face k)
    fzz = (0.5 * (w[:-1] + w[1:])) ** 2                       # centre k
    au = (_x(fxx, 1) - fxx) / g.dx + (fxy - _y(fxy, -1)) / g.dy + (fxz[1:] - fxz[:-1]) / _col(g.dzf)
    av = (fxy - _x(fxy, -1)) / g.dx + (_y(fyy, 1) - fyy) / g.dy + (fyz[1:] - fyz[:-1]) / _col(g.dzf)
    aw = np.zeros_like(w)
    aw[1:-1] = ((fxz[1:-1] - _x(fxz[1:-1], -1)) / g.dx + (fyz[1:-1] - _y(fyz[1:-1], -1)) / g.dy
                + (fzz[1:] - fzz[:-1]) / _col(g.dzc[1:-1]))
    return au, av, aw


def viscous(u, v, w, g: Grid):
    """The Laplacian L of each staggered component (no-slip ghosts for u, v;
    w on the interior faces, zero rows at the walls)."""
    out = []
    for c in (u, v):
        ce = _ghost(c, -1.0)
        lz = ((ce[2:] - ce[1:-1]) / _col(g.dzc[1:]) - (ce[1:-1] - ce[:-2]) / _col(g.dzc[:-1])) / _col(g.dzf)
        out.append((_x(c, 1) - 2 * c + _x(c, -1)) / g.dx ** 2 + (_y(c, 1) - 2 * c + _y(c, -1)) / g.dy ** 2 + lz)
    lw = np.zeros_like(w)
    wi = w[1:-1]
    lw[1:-1] = ((_x(wi, 1) - 2 * wi + _x(wi, -1)) / g.dx ** 2 + (_y(wi, 1) - 2 * wi + _y(wi, -1)) / g.dy ** 2
                + ((w[2:] - w[1:-1]) / _col(g.dzf[1:]) - (w[1:-1] - w[:-2]) / _col(g.dzf[:-1]))
                / _col(g.dzc[1:-1]))
    out.append(lw)
    return out


def sgs_divergence(u, v, w, nut, g: Grid):
    """d(2 nu_t S_ij)/dx_j at the u, v, w points (T1, T3, T4)."""
    ue, ve, ne = _ghost(u, -1.0), _ghost(v, -1.0), _ghost(nut, 1.0)
    t11 = 2 * nut * (u - _x(u, -1)) / g.dx                    # centres
    t22 = 2 * nut * (v - _y(v, -1)) / g.dy
    t33 = 2 * nut * (w[1:] - w[:-1]) / _col(g.dzf)
    n12 = 0.25 * (nut + _x(nut, 1) + _y(nut, 1) + _x(_y(nut, 1), 1))
    t12 = 2 * n12 * 0.5 * ((_y(u, 1) - u) / g.dy + (_x(v, 1) - v) / g.dx)          # edge (i+1/2, j+1/2)
    n13 = 0.25 * (ne[:-1] + ne[1:] + _x(ne[:-1], 1) + _x(ne[1:], 1))
    t13 = 2 * n13 * 0.5 * ((ue[1:] - ue[:-1]) / _col(g.dzc) + (_x(w, 1) - w) / g.dx)  # edge (i+1/2, face k)
    n23 = 0.25 * (ne[:-1] + ne[1:] + _y(ne[:-1], 1) + _y(ne[1:], 1))
    t23 = 2 * n23 * 0.5 * ((ve[1:] - ve[:-1]) / _col(g.dzc) + (_y(w, 1) - w) / g.dy)  # edge (j+1/2, face k)
    du = (_x(t11, 1) - t11) / g.dx + (t12 - _y(t12, -1)) / g.dy + (t13[1:] - t13[:-1]) / _col(g.dzf)
    dv = (t12 - _x(t12, -1)) / g.dx + (_y(t22, 1) - t22) / g.dy + (t23[1:] - t23[:-1]) / _col(g.dzf)
    dw = np.zeros_like(w)
    dw[1:-1] = ((t13[1:-1] - _x(t13[1:-1], -1)) / g.dx + (t23[1:-1] - _y(t23[1:-1], -1)) / g.dy
                + (t33[1:] - t33[:-1]) / _col(g.dzc[1:-1]))
    return du, dv, dw


def momentum_rhs(u, v, w, nut, g: Grid, nu: float):
    """R = H + nu L u = -advection + nu L u + d(2 nu_t S_ij)/dx_j (T1)."""
    adv = advection(u, v, w, g)
    lap = viscous(u, v, w, g)
    sgs = sgs_divergence(u, v, w, nut, g)
    return [-a + nu * l + s for a, l, s in zip(adv, lap, sgs)]


def rk3_substep(u, v, w, p, nut, r_prev, g: Grid, stage: int, dt: float, nu: float, cs: float, utau: float):
    """One substep (stage 0, 1, 2) of Eqs. 11-14 and the nu_t update.

    r_prev is R^{k-1} (ignored at stage 0, where beta = 0).  Returns
    (u, v, w, p, nut, R^k) of the next substep."""
    a, b, gm = RK3_ALPHA[stage], RK3_BETA[stage], RK3_GAMMA[stage]
    r = momentum_rhs(u, v, w, nut, g, nu)
    gp = gradient(p, g)
    star = []
    for c, rc, rp, gc in zip((u, v, w), r, r_prev if b != 0.0 else (None,) * 3, gp):
        inc = a * rc - gm * gc
        if b != 0.0:
            inc = inc + b * rp
        star.append(c + dt * inc)
    star[2][0] = 0.0
    star[2][-1] = 0.0
    # L phi' = div u*; phi = phi' / (gamma dt); u = u* - gamma dt grad phi = u* - grad phi'
    phi_s = solve(divergence(*star, g), g)
    gx, gy, gz = gradient(phi_s, g)
    un, vn, wn = star[0] - gx, star[1] - gy, star[2] - gz
    pn = p + phi_s / (gm * dt)
    nutn = eddy_viscosity(un, vn, wn, g, cs, nu, utau)
    return un, vn, wn, pn, nutn, r
