"""Pins of the eddy-viscosity oracle (Eq. 4 with van Driest damping), no GPU:
closed forms of discrete linear fields, the zero-strain limit, second-order
convergence of |S| to the continuous strain rate, and the damping limits."""
import math

import numpy as np
import pytest

import oracle as O
import synth_inputs as S


def grid(nx, ny, nz, beta=1.6, lx=2 * math.pi, ly=math.pi, lz=2.0):
    dzc, dzf = O.cell_spacings(S.tanh_faces(nz, beta, lz))
    return O.Grid(nx, ny, nz, lx / nx, ly / ny, dzc, dzf, (0, 0, 0, 0, 2, 2))


def centres_z(g):
    zf = np.concatenate([[0.0], np.cumsum(g.dzf)])
    return 0.5 * (zf[:-1] + zf[1:]), zf


def test_linear_shear_has_closed_form_strain_away_from_walls():
    g = grid(8, 6, 20)
    zc, zf = centres_z(g)
    a = 3.7
    u = np.broadcast_to((a * zc).reshape(-1, 1, 1), (20, 6, 8)).copy()   # u = a z: du/dz exact on any grid
    v = np.zeros_like(u)
    w = np.zeros((21, 6, 8))
    s11, s22, s33, s12, s13, s23 = O.strain_rate(u, v, w, g)
    # interior cells (both z-faces interior): S13 = a/2 exactly, the rest zero
    assert np.allclose(s13[1:-1], a / 2, rtol=1e-13) and np.allclose(s12, 0) and np.allclose(s23, 0)
    assert np.allclose(s11, 0) and np.allclose(s22, 0) and np.allclose(s33, 0)
    nut = O.eddy_viscosity(u, v, w, g, 0.1, 1e-3, 0.05)
    coef = (0.1 * np.cbrt(g.dx * g.dy * g.dzf) * O.van_driest(g, 1e-3, 0.05)) ** 2
    assert np.allclose(nut[1:-1], (coef[1:-1] * abs(a)).reshape(-1, 1, 1), rtol=1e-13)


def test_uniform_translation_has_no_interior_strain():
    g = grid(8, 8, 12)
    u = np.full((12, 8, 8), 1.3)
    v = np.full((12, 8, 8), -0.4)
    w = np.zeros((13, 8, 8))
    nut = O.eddy_viscosity(u, v, w, g, 0.17, 1e-3, 0.05)
    assert np.all(nut[1:-1] == 0.0) and np.all(nut[0] > 0) and np.all(nut[-1] > 0)   # only the no-slip wall layers


def _smooth(g):
    """u, v, w samples of a smooth field (periodic in x, y; u = v = w = 0 on the
    walls) and the exact 2 S_ij S_ij at the cell centres."""
    lx, ly = g.nx * g.dx, g.ny * g.dy
    zc, zf = centres_z(g)
    x_c = (np.arange(g.nx) + 0.5) * g.dx
    x_f = (np.arange(g.nx) + 1.0) * g.dx
    y_c = (np.arange(g.ny) + 0.5) * g.dy
    y_f = (np.arange(g.ny) + 1.0) * g.dy
    kx, ky = 2 * np.pi / lx, 2 * np.pi / ly
    # u = sin(kx x) cos(ky y) h(z), v = cos(kx x) sin(ky y) h(z), w = sin(kx x) sin(ky y) q(z)
    h = lambda z: np.sin(np.pi * z / zf[-1])                       # zero at the walls (no slip)
    dh = lambda z: np.pi / zf[-1] * np.cos(np.pi * z / zf[-1])
    q = lambda z: np.sin(np.pi * z / zf[-1]) ** 2
    dq = lambda z: np.pi / zf[-1] * np.sin(2 * np.pi * z / zf[-1])
    Z, Y, X = np.meshgrid(zc, y_c, x_f, indexing="ij"); u = np.sin(kx * X) * np.cos(ky * Y) * h(Z)
    Z, Y, X = np.meshgrid(zc, y_f, x_c, indexing="ij"); v = np.cos(kx * X) * np.sin(ky * Y) * h(Z)
    Z, Y, X = np.meshgrid(zf, y_c, x_c, indexing="ij"); w = np.sin(kx * X) * np.sin(ky * Y) * q(Z)
    Z, Y, X = np.meshgrid(zc, y_c, x_c, indexing="ij")
    s11 = kx * np.cos(kx * X) * np.cos(ky * Y) * h(Z)
    s22 = ky * np.cos(kx * X) * np.cos(ky * Y) * h(Z)
    s33 = np.sin(kx * X) * np.sin(ky * Y) * dq(Z)
    s12 = 0.5 * (-ky * np.sin(kx * X) * np.sin(ky * Y) * h(Z) - kx * np.sin(kx * X) * np.sin(ky * Y) * h(Z))
    s13 = 0.5 * (np.sin(kx * X) * np.cos(ky * Y) * dh(Z) + kx * np.cos(kx * X) * np.sin(ky * Y) * q(Z))
    s23 = 0.5 * (np.cos(kx * X) * np.sin(ky * Y) * dh(Z) + ky * np.sin(kx * X) * np.cos(ky * Y) * q(Z))
    s2 = 2 * (s11 ** 2 + s22 ** 2 + s33 ** 2 + 2 * (s12 ** 2 + s13 ** 2 + s23 ** 2))
    return u, v, w, s2


def test_strain_rate_converges_at_second_order():
    errs = []
    for n in (16, 32, 64):
        g = O.Grid(n, n, n, 2 * math.pi / n, math.pi / n, np.full(n + 1, 2.0 / n), np.full(n, 2.0 / n),
                   (0, 0, 0, 0, 2, 2))                         # uniform z: centred differences everywhere inside
        u, v, w, s2 = _smooth(g)
        c = O.strain_rate(u, v, w, g)
        got = 2 * (c[0] ** 2 + c[1] ** 2 + c[2] ** 2 + 2 * (c[3] ** 2 + c[4] ** 2 + c[5] ** 2))
        inner = slice(n // 4, 3 * n // 4)                     # away from the walls' one-sided ghost stencils
        errs.append(np.abs(got[inner] - s2[inner]).max() / np.abs(s2[inner]).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r > 1.8 for r in rates), (errs, rates)


def test_van_driest_limits():
    g = grid(4, 4, 64, beta=2.0)
    d = O.van_driest(g, 1e-4, 0.05)                           # Re_tau = 500 on half-height 1
    zc, zf = centres_z(g)
    dist = np.minimum(zc, zf[-1] - zc)
    assert np.all((d > 0) & (d < 1))
    assert np.allclose(d, 1 - np.exp(-dist * 0.05 / 1e-4 / 25.0))
    assert d[0] < 0.1 and d[g.nz // 2] > 0.999 and abs(d[0] - d[-1]) < 1e-12   # symmetric tanh grid
