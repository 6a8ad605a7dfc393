"""Pins of the oracle's periodic-z solve (cyclic tridiagonal per mode): dense
LU of the whole staggered operator, closed-form discrete eigenfunctions,
the singular all-periodic case, and a planted mistake."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.cales_oracle as C
import synth_inputs as S


def periodic_grid(nx, ny, nz, bcx, bcy, beta, lz=2.0):
    """Stretched periodic z: the wrap distance dzc[0] = dzc[nz] joins the last
    cell centre to the first through the period."""
    zf = S.tanh_faces(nz, beta, lz) if beta > 0 else np.linspace(0.0, lz, nz + 1)
    dzc, dzf = O.cell_spacings(zf)
    dzc[0] = dzc[-1] = 0.5 * (dzf[0] + dzf[-1])
    return O.Grid(nx, ny, nz, 2 * math.pi / nx, 1.3 / ny, dzc, dzf, (bcx, bcx, bcy, bcy, O.BC_P, O.BC_P))


@pytest.mark.parametrize("bcx,bcy", [(O.BC_P, O.BC_P), (O.BC_P, O.BC_N), (O.BC_N, O.BC_D), (O.BC_D, O.BC_P)])
@pytest.mark.parametrize("alpha", [None, 0.03])
def test_periodic_z_matches_dense_lu(bcx, bcy, alpha):
    g = periodic_grid(6, 4, 7, bcx, bcy, 1.6)
    f = S.gaussian(500 + bcx * 7 + bcy, (g.nz, g.ny, g.nx))
    if O.is_singular(g, alpha):
        f = O.project(f, g)
    assert O.rel_l2(O.solve(f, g, alpha), O.dense_solve(f, g, alpha)) < 1e-11


@pytest.mark.parametrize("mz", [1, 3])
def test_periodic_z_eigenfunctions(mz):
    """Uniform periodic grid: cos(2 pi (mx i / nx + mz k / nz)) has the
    eigenvalue -4/dx^2 sin^2(pi mx/nx) - 4/dz^2 sin^2(pi mz/nz) (Helmholtz form)."""
    g = periodic_grid(8, 4, 10, O.BC_P, O.BC_P, 0.0)
    mx = 2
    i, k = np.arange(g.nx), np.arange(g.nz)
    p = np.cos(2 * np.pi * (mx * i[None, None, :] / g.nx + mz * k[:, None, None] / g.nz)) * np.ones((1, g.ny, 1))
    lam = -4 / g.dx ** 2 * np.sin(np.pi * mx / g.nx) ** 2 - 4 / g.dzf[0] ** 2 * np.sin(np.pi * mz / g.nz) ** 2
    assert np.max(np.abs(O.apply_L(p, g) - lam * p)) < 1e-11 * abs(lam)
    alpha = 0.2
    assert np.max(np.abs(O.solve((1 - alpha * lam) * p, g, alpha) - p)) < 1e-12


def test_periodic_z_singular_poisson_is_projected_and_gauged():
    g = periodic_grid(8, 6, 9, O.BC_P, O.BC_N, 1.4)
    f = S.gaussian(520, (g.nz, g.ny, g.nx))                 # not consistent: the solve projects it
    p = O.solve(f, g)
    assert abs(O.weighted_mean(p, g)) < 1e-13
    assert O.rel_l2(O.apply_L(p, g), O.project(f, g)) < 1e-11


def test_mutation_dropped_corners_fail_the_dense_pin(monkeypatch):
    monkeypatch.setattr(C, "cyclic_solve", C.thomas)
    with pytest.raises(AssertionError):
        test_periodic_z_matches_dense_lu(O.BC_P, O.BC_N, 0.03)


@pytest.mark.parametrize("bcx,bcy", [(O.BC_P, O.BC_P), (O.BC_N, O.BC_D)])
@pytest.mark.parametrize("alpha", [None, 0.03])
def test_periodic_z_transpose_matches_dense(bcx, bcy, alpha):
    """The transposed solve over a periodic z (corners swapped) is the dense
    transpose of the solve map, assembled column by column."""
    g = periodic_grid(4, 3, 6, bcx, bcy, 1.5)
    n = g.nx * g.ny * g.nz
    smat = np.empty((n, n))
    e = np.zeros(n)
    for q in range(n):
        e[q] = 1.0
        smat[:, q] = O.solve(e.reshape(g.nz, g.ny, g.nx), g, alpha).reshape(-1)
        e[q] = 0.0
    w = S.gaussian(530 + bcx, (g.nz, g.ny, g.nx))
    assert O.rel_l2(O.solve_T(w, g, alpha), (smat.T @ w.reshape(-1)).reshape(w.shape)) < 1e-11


@pytest.mark.parametrize("alpha", [1e-3, 0.2])
def test_periodic_z_line_solves_against_the_stencil(alpha):
    """(I - alpha L_z) u = f on each (i, j) line with the wrap coupling: the
    z part of the stencil applied to the result returns f."""
    g = periodic_grid(5, 3, 8, O.BC_P, O.BC_P, 1.5)
    f = S.gaussian(540, (g.nz, g.ny, g.nx))
    u = O.solve_z_lines(f, g, alpha)
    zm, zp = np.roll(u, 1, axis=0), np.roll(u, -1, axis=0)
    dzc = g.dzc.reshape(-1, 1, 1)
    dzf = g.dzf.reshape(-1, 1, 1)
    lz = ((zp - u) / dzc[1:] - (u - zm) / dzc[:-1]) / dzf
    assert np.max(np.abs(u - alpha * lz - f)) < 1e-12 * np.max(np.abs(f))
