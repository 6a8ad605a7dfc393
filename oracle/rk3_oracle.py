"""FP64 oracle of the explicit low-storage RK3 pressure-correction substep.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2, Eqs. 11-14 with the explicit viscous term (Algorithm 1):
    u*        = u^k + dt [alpha (H^k + nu L u^k) + beta (H^{k-1} + nu L u^{k-1}) - gamma grad p^{k-1/2}]
    L phi     = div u* / (gamma dt)
    u^{k+1}   = u* - gamma dt grad phi
    p^{k+1/2} = p^{k-1/2} + phi
followed by nu_t^{k+1} from u^{k+1} (Eq. 4).  alpha, beta, gamma are the
Wray coefficients printed below Eq. 14.  Crank-Nicolson variants:
  implicit = 1 (Eqs. 17-19): u** = u^k + dt [alpha H^k + beta H^{k-1} + gamma (nu L u^k - grad p)],
      (1 - gamma nu dt/2 L) u* = u** - gamma nu dt/2 L u^k (modified Helmholtz, Eq. 18),
      p^{k+1/2} = p^{k-1/2} + phi - gamma nu dt/2 L phi;
  implicit = 2 (Eqs. 20-22): the same with only the wall-normal part L_z
      implicit; nu (L_x + L_y) u stays with H in the explicit RK3 terms.
The paper leaves open, read here as:

T1  signs of H_i (Eq. 15) from the momentum equation (Eq. 2) and the
    Boussinesq closure (Eq. 3): H_i = -d(u_i u_j)/dx_j + d(2 nu_t S_ij)/dx_j;
    the right-hand side carried between substeps is R = H + nu L u;
T2  advection in divergence form on the staggered grid, every interpolated
    velocity the arithmetic mean of its two neighbours (also in stretched z);
T3  channel: x, y periodic, no-slip walls in z (u, v ghosts minus the first
    interior value at the distances dzc[0], dzc[nz]; w = 0 on the wall faces);
    strain rates as the eddy-viscosity oracle forms them on cell edges;
T4  nu_t on an edge is the mean of the four cell centres around it; beyond a
    wall the ghost centre repeats the first interior value;
T6  the implicit solves take the velocity's own wall conditions: u and v are
    cell-centred Dirichlet (the no-slip ghost), w is node-centred on the
    interior faces with w = 0 on the walls; L phi in the pressure update
    takes the pressure's Neumann walls.

Layout as the rest of the oracle: u [nz][ny][nx] on x-faces i+1/2, v on
y-faces j+1/2, w [nz+1][ny][nx] on z-faces, p, nu_t at cell centres.
"""
from __future__ import annotations

import numpy as np

from .cales_oracle import BC_D, BC_DF, Grid, divergence, gradient, solve, solve_z_lines
from .sgs_oracle import eddy_viscosity

__all__ = ["RK3_ALPHA", "RK3_BETA", "RK3_GAMMA", "advection", "viscous", "viscous_parts", "sgs_divergence",
           "momentum_rhs", "velocity_grids", "laplacian_cell", "rk3_rhs", "rk3_substep"]

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


def _lxy(c, g: Grid):
    return (_x(c, 1) - 2 * c + _x(c, -1)) / g.dx ** 2 + (_y(c, 1) - 2 * c + _y(c, -1)) / g.dy ** 2


def _lz_cell(c, g: Grid, sign):
    """z part of the Laplacian of a cell-centred field, ghosts sign * first value."""
    ce = _ghost(c, sign)
    return ((ce[2:] - ce[1:-1]) / _col(g.dzc[1:]) - (ce[1:-1] - ce[:-2]) / _col(g.dzc[:-1])) / _col(g.dzf)


def viscous_parts(u, v, w, g: Grid):
    """(L_x + L_y, L_z) of each staggered component (no-slip ghosts for u, v;
    w on the interior faces, zero rows at the walls)."""
    out = [(_lxy(c, g), _lz_cell(c, g, -1.0)) for c in (u, v)]
    lxy, lz = np.zeros_like(w), np.zeros_like(w)
    lxy[1:-1] = _lxy(w[1:-1], g)
    lz[1:-1] = ((w[2:] - w[1:-1]) / _col(g.dzf[1:]) - (w[1:-1] - w[:-2]) / _col(g.dzf[:-1])) / _col(g.dzc[1:-1])
    out.append((lxy, lz))
    return out


def viscous(u, v, w, g: Grid):
    """The Laplacian L of each staggered component."""
    return [a + b for a, b in viscous_parts(u, v, w, g)]


def laplacian_cell(phi, g: Grid, z_only=False):
    """L (or L_z) of a cell-centred scalar with Neumann z walls (the pressure)."""
    lz = _lz_cell(phi, g, 1.0)
    return lz if z_only else _lxy(phi, g) + lz


def velocity_grids(g: Grid):
    """Grids of the implicit velocity solves (T6): u, v cell-centred with
    Dirichlet walls; w on the interior faces 1..nz-1 with wall nodes."""
    guv = Grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dzc, g.dzf, (0, 0, 0, 0, BC_D, BC_D))
    gw = Grid(g.nx, g.ny, g.nz - 1, g.dx, g.dy, g.dzf, g.dzc[1:-1], (0, 0, 0, 0, BC_DF, BC_DF))
    return guv, gw


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


def rk3_rhs(u, v, w, p, nut, r_prev, g: Grid, stage: int, dt: float, nu: float, implicit: int = 0):
    """Right-hand side of the velocity update of one substep and the term
    carried to the next (R^k).  implicit = 0: u* itself (Eq. 11), R = H + nu L u;
    1: u** - gamma nu dt/2 L u^k (Eqs. 17-18), R = H; 2: the same with L_z,
    R = H + nu (L_x + L_y) u (Eqs. 20-21)."""
    a, b, gm = RK3_ALPHA[stage], RK3_BETA[stage], RK3_GAMMA[stage]
    adv = advection(u, v, w, g)
    parts = viscous_parts(u, v, w, g)
    sgs = sgs_divergence(u, v, w, nut, g)
    gp = gradient(p, g)
    rhs, carry = [], []
    for c, ac, (lxy, lz), sc, gc, rp in zip((u, v, w), adv, parts, sgs, gp,
                                             r_prev if b != 0.0 else (None,) * 3):
        h = -ac + sc
        if implicit == 0:
            r = h + nu * (lxy + lz)
            inc = a * r - gm * gc
        elif implicit == 1:
            r = h
            inc = a * r - gm * gc + gm * nu * (lxy + lz)
        else:
            r = h + nu * lxy
            inc = a * r - gm * gc + gm * nu * lz
        if b != 0.0:
            inc = inc + b * rp
        star = c + dt * inc
        if implicit == 1:
            star = star - gm * nu * dt / 2 * (lxy + lz)
        elif implicit == 2:
            star = star - gm * nu * dt / 2 * lz
        rhs.append(star)
        carry.append(r)
    rhs[2][0] = 0.0
    rhs[2][-1] = 0.0
    return rhs, carry


def rk3_substep(u, v, w, p, nut, r_prev, g: Grid, stage: int, dt: float, nu: float, cs: float, utau: float,
                implicit: int = 0):
    """One substep (stage 0, 1, 2): Eqs. 11-14 (implicit = 0), Eqs. 17-19
    (implicit = 1) or Eqs. 20-22 (implicit = 2), then the nu_t update.

    r_prev is R^{k-1} (ignored at stage 0, where beta = 0).  Returns
    (u, v, w, p, nut, R^k) of the next substep."""
    gm = RK3_GAMMA[stage]
    star, r = rk3_rhs(u, v, w, p, nut, r_prev, g, stage, dt, nu, implicit)
    ah = gm * nu * dt / 2
    if implicit:
        guv, gw = velocity_grids(g)
        sol = solve if implicit == 1 else solve_z_lines
        ws = np.zeros_like(star[2])
        ws[1:-1] = sol(star[2][1:-1], gw, ah)
        star = [sol(star[0], guv, ah), sol(star[1], guv, ah), ws]
    # L phi' = div u*; phi = phi' / (gamma dt); u = u* - gamma dt grad phi = u* - grad phi'
    phi_s = solve(divergence(*star, g), g)
    gx, gy, gz = gradient(phi_s, g)
    un, vn, wn = star[0] - gx, star[1] - gy, star[2] - gz
    phi = phi_s / (gm * dt)
    if implicit:
        phi = phi - ah * laplacian_cell(phi, g, z_only=implicit == 2)
    pn = p + phi
    nutn = eddy_viscosity(un, vn, wn, g, cs, nu, utau)
    return un, vn, wn, pn, nutn, r
