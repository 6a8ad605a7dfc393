"""Pins of the FP64 oracle against facts fixed by the mathematics (no GPU).

Each test ties the oracle to something other than itself: closed-form
discrete eigenfunctions, library transforms (numpy/scipy FFT, DCT, DST),
LAPACK dense LU, LAPACK banded solves, second-order convergence to the
continuous Laplacian, and transpose identities.  The mutation tests at the
end plant plausible mistakes in a copy of the oracle and check that a pin
catches each one.
"""
import itertools
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle as O
import synth_inputs as S

RNG = np.random.default_rng(20241114)
KINDS_XY = (O.BC_P, O.BC_N, O.BC_D)
KINDS_Z = (O.BC_N, O.BC_D, O.BC_DF)


def make_grid(nx, ny, nz, bc, beta=1.4, lx=2 * math.pi, ly=math.pi, lz=2.0):
    if beta is None:
        dzc = np.full(nz + 1, lz / nz)
        dzf = np.full(nz, lz / nz)
    elif bc[4] == O.BC_DF or bc[5] == O.BC_DF:
        dzc, dzf = O.face_spacings(S.tanh_faces(nz + 1, beta, lz))
    else:
        dzc, dzf = O.cell_spacings(S.tanh_faces(nz, beta, lz))
    return O.Grid(nx, ny, nz, lx / nx, ly / ny, dzc, dzf, bc)


# ---------------------------------------------------------------------------
# transforms against library routines and closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 30])
def test_transforms_match_library(n):
    x = RNG.standard_normal(n)
    assert np.allclose(O.fwd_matrix(O.BC_P, n) @ x, np.fft.fft(x), atol=1e-12)
    # scipy's unnormalised DCT-II / DST-II carry a factor 2
    assert np.allclose(O.fwd_matrix(O.BC_N, n) @ x, scipy.fft.dct(x, type=2) / 2, atol=1e-12)
    assert np.allclose(O.fwd_matrix(O.BC_D, n) @ x, scipy.fft.dst(x, type=2) / 2, atol=1e-12)
    for k in KINDS_XY:
        assert np.allclose(O.inv_matrix(k, n) @ (O.fwd_matrix(k, n) @ x), x, atol=1e-12)


def _second_difference(kind, n, h):
    """1-D second difference with the R2 ghost rules, built entry by entry."""
    d = np.zeros((n, n))
    for i in range(n):
        d[i, i] -= 2.0
        for nb in (i - 1, i + 1):
            if 0 <= nb < n:
                d[i, nb] += 1.0
            elif kind == O.BC_P:
                d[i, nb % n] += 1.0
            elif kind == O.BC_N:
                d[i, i] += 1.0
            elif kind == O.BC_D:
                d[i, i] -= 1.0
    return d / h ** 2


@pytest.mark.parametrize("kind", KINDS_XY)
@pytest.mark.parametrize("n", [1, 2, 4, 7, 16])
def test_transform_diagonalises_second_difference(kind, n):
    h = 0.37
    fm = O.fwd_matrix(kind, n)
    lam = O.eigenvalues(kind, n, h)
    d2 = _second_difference(kind, n, h)
    assert np.allclose(fm @ d2, lam[:, None] * fm, atol=1e-9 * np.abs(lam).max() + 1e-12)


# ---------------------------------------------------------------------------
# analytic discrete eigenfunctions on a uniform grid
# ---------------------------------------------------------------------------
def _basis_xy(kind, n, m):
    i = np.arange(n)
    if kind == O.BC_P:
        return np.cos(2 * math.pi * m * i / n), -(4 / 1.0) * math.sin(math.pi * m / n) ** 2
    if kind == O.BC_N:
        return np.cos(math.pi * m * (i + 0.5) / n), -4 * math.sin(math.pi * m / (2 * n)) ** 2
    return np.sin(math.pi * m * (i + 0.5) / n), -4 * math.sin(math.pi * m / (2 * n)) ** 2


def _basis_z(kind, n, m):
    k = np.arange(n)
    if kind == O.BC_N:
        return np.cos(math.pi * m * (k + 0.5) / n), -4 * math.sin(math.pi * m / (2 * n)) ** 2
    if kind == O.BC_D:
        return np.sin(math.pi * m * (k + 0.5) / n), -4 * math.sin(math.pi * m / (2 * n)) ** 2
    return np.sin(math.pi * m * (k + 1) / (n + 1)), -4 * math.sin(math.pi * m / (2 * (n + 1))) ** 2


@pytest.mark.parametrize("kx,ky,kz", list(itertools.product(KINDS_XY, KINDS_XY, KINDS_Z)))
@pytest.mark.parametrize("alpha", [None, 3e-3])
def test_discrete_eigenfunctions(kx, ky, kz, alpha):
    nx, ny, nz = 12, 10, 9
    dx, dy, dz = 0.5, 0.25, 0.2
    g = O.Grid(nx, ny, nz, dx, dy, np.full(nz + 1, dz), np.full(nz, dz), (kx, kx, ky, ky, kz, kz))
    for a, b, c in [(1, 2, 1), (3, 1, 2), (2, 4, 3)]:
        px, lx = _basis_xy(kx, nx, a)
        py, ly = _basis_xy(ky, ny, b)
        pz, lz = _basis_z(kz, nz, c)
        lam = lx / dx ** 2 + ly / dy ** 2 + lz / dz ** 2
        pstar = pz[:, None, None] * py[None, :, None] * px[None, None, :]
        f = lam * pstar if alpha is None else (1 - alpha * lam) * pstar
        assert np.allclose(O.apply_M(pstar, g, alpha), f, atol=1e-10 * np.abs(f).max())
        p = O.solve(f, g, alpha)
        assert O.rel_l2(p, pstar) < 1e-13


# ---------------------------------------------------------------------------
# dense LU on every boundary combination (stretched z, odd sizes)
# ---------------------------------------------------------------------------
DENSE_CASES = list(itertools.product(KINDS_XY, KINDS_XY, KINDS_Z, KINDS_Z))


@pytest.mark.parametrize("kx,ky,zlo,zhi", DENSE_CASES)
def test_dense_lu(kx, ky, zlo, zhi):
    bc = (kx, kx, ky, ky, zlo, zhi)
    for (nx, ny, nz), alpha in [((5, 3, 7), None), ((4, 6, 5), 2e-2), ((8, 8, 8), None)]:
        if nx * ny * nz > 300 and (zlo, zhi) != (O.BC_N, O.BC_N):
            continue
        g = make_grid(nx, ny, nz, bc)
        f = RNG.standard_normal((nz, ny, nx))
        assert O.rel_l2(O.solve(f, g, alpha), O.dense_solve(f, g, alpha)) < 1e-12


def test_dense_lu_8cubed_all_walls():
    g = make_grid(8, 8, 8, (O.BC_D, O.BC_D, O.BC_N, O.BC_N, O.BC_D, O.BC_DF))
    f = RNG.standard_normal((8, 8, 8))
    assert O.rel_l2(O.solve(f, g), O.dense_solve(f, g)) < 1e-12


# ---------------------------------------------------------------------------
# the stencil converges to the continuous Laplacian (pins dzc/dzf roles)
# ---------------------------------------------------------------------------
def test_second_order_convergence_stretched():
    """Interior truncation error and the solution error both fall as h^2.

    (In the wall cell the cell-centred truncation error is only first order;
    the solution still converges at second order.)
    """
    terr, serr = [], []
    for n in (16, 32, 64):
        g = make_grid(4, 4, n, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_N, O.BC_N), beta=1.8,
                      lx=2 * math.pi, ly=2 * math.pi)
        zf = S.tanh_faces(n, 1.8)
        zc = 0.5 * (zf[1:] + zf[:-1])
        x = np.arange(4) * g.dx
        pz = np.cos(math.pi * zc)          # dp/dz = 0 at z = 0 and 2
        p = pz[:, None, None] * np.cos(x)[None, None, :] * np.ones((1, 4, 1))
        exact = -(math.pi ** 2) * p + (2 * (np.cos(g.dx) - 1) / g.dx ** 2) * p
        inner = slice(n // 4, 3 * n // 4)
        terr.append(np.abs((O.apply_L(p, g) - exact)[inner]).max())
        serr.append(np.abs(O.solve(exact, g) - p).max())
    assert terr[0] / terr[1] > 3.2 and terr[1] / terr[2] > 3.2
    assert serr[0] / serr[1] > 3.2 and serr[1] / serr[2] > 3.2


def test_second_order_convergence_face_unknowns():
    errs = []
    for n in (16, 32, 64):
        zf = S.tanh_faces(n, 1.5)
        dzc, dzf = O.face_spacings(zf)
        g = O.Grid(1, 1, n - 1, 1.0, 1.0, dzc, dzf, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_DF, O.BC_DF))
        z = zf[1:-1]
        p = np.sin(math.pi * z / 2).reshape(-1, 1, 1)       # zero at z = 0 and 2
        exact = -(math.pi / 2) ** 2 * p
        errs.append(np.abs(O.apply_L(p, g) - exact).max())
    assert errs[0] / errs[1] > 3.2 and errs[1] / errs[2] > 3.2


# ---------------------------------------------------------------------------
# residuals, symmetry, transposes, reductions to simpler problems
# ---------------------------------------------------------------------------
def test_residual_machine_precision_channel():
    g = make_grid(64, 32, 32, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_N, O.BC_N), beta=None)
    f = S.remove_mean(S.uniform(1000, (32, 32, 64)))
    p = O.solve(f, g)
    assert O.rel_l2(O.apply_L(p, g), f) < 1e-13
    assert abs(O.weighted_mean(p, g)) < 1e-15 * np.abs(p).max()


@pytest.mark.parametrize("alpha", [None, 1e-3])
def test_residual_machine_precision_stretched_duct(alpha):
    g = make_grid(24, 16, 20, (O.BC_P, O.BC_P, O.BC_N, O.BC_N, O.BC_N, O.BC_N), beta=1.5)
    f = S.gaussian(7, (20, 16, 24))
    p = O.solve(f, g, alpha)
    rhs = O.project(f, g) if alpha is None else f
    assert O.rel_l2(O.apply_M(p, g, alpha), rhs) < 1e-13


@pytest.mark.parametrize("alpha", [None, 1e-4])
def test_refined_solve_reaches_the_exact_discrete_solution(alpha):
    """Deep stretched z (the benchmark's 512 cells, tanh 1.5): a smooth p*
    (the solution of a Gaussian right-hand side) and f = M p* by the stencil;
    the refined solve returns p* at the stencil's rounding floor, where the
    plain expansion is off by cond * eps (about 1e-12).  On a grid small
    enough for dense LU the two agree with LAPACK."""
    g = make_grid(64, 32, 512, (O.BC_P, O.BC_P, O.BC_N, O.BC_N, O.BC_N, O.BC_N), beta=1.5, lx=6.0, ly=2.0)
    p_star = O.solve(S.gaussian(3001, (512, 32, 64)), g, alpha)
    f = O.apply_M(p_star, g, alpha)
    plain, refined = O.solve(f, g, alpha), O.solve_refined(f, g, alpha)
    assert O.rel_l2(refined, p_star) < 1e-14, O.rel_l2(refined, p_star)
    assert O.rel_l2(refined, p_star) < O.rel_l2(plain, p_star)
    gs = make_grid(6, 4, 8, (O.BC_P, O.BC_P, O.BC_N, O.BC_N, O.BC_N, O.BC_D), beta=1.5)
    fs = S.gaussian(3002, (8, 4, 6))
    assert O.rel_l2(O.solve_refined(fs, gs, alpha), O.dense_solve(fs, gs, alpha)) < 1e-13


def test_weighted_symmetry():
    g = make_grid(6, 5, 7, (O.BC_N, O.BC_N, O.BC_D, O.BC_D, O.BC_D, O.BC_N), beta=1.7)
    p, q = RNG.standard_normal((2, 7, 5, 6))
    w = g.dzf.reshape(-1, 1, 1)
    assert np.isclose((O.apply_L(p, g) * q * w).sum(), (p * O.apply_L(q, g) * w).sum(), rtol=1e-12)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0, 1, 1), (0, 0, 1, 1, 1, 1), (2, 2, 0, 0, 2, 3)])
@pytest.mark.parametrize("alpha", [None, 1e-2])
def test_transpose_matches_dense(bc, alpha):
    g = make_grid(4, 3, 5, bc)
    n = 60
    smat = np.empty((n, n))
    e = np.zeros(n)
    for q in range(n):
        e[q] = 1
        smat[:, q] = O.solve(e.reshape(5, 3, 4), g, alpha).reshape(-1)
        e[q] = 0
    w = RNG.standard_normal((5, 3, 4))
    assert np.allclose(O.solve_T(w, g, alpha).reshape(-1), smat.T @ w.reshape(-1), atol=1e-11)


def test_one_dimensional_reduction_banded():
    nz = 40
    g = make_grid(1, 1, nz, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_D, O.BC_N), beta=2.0)
    f = RNG.standard_normal((nz, 1, 1))
    sub, diag, sup = O.z_operator(g)
    ab = np.zeros((3, nz))
    ab[0, 1:] = sup[:-1]
    ab[1] = diag
    ab[2, :-1] = sub[1:]
    ref = scipy.linalg.solve_banded((1, 1), ab, f.reshape(-1))
    assert O.rel_l2(O.solve(f, g).reshape(-1), ref) < 1e-13


def test_shift_equivariance_periodic_x():
    g = make_grid(16, 8, 6, (O.BC_P, O.BC_P, O.BC_N, O.BC_N, O.BC_D, O.BC_D))
    f = RNG.standard_normal((6, 8, 16))
    assert np.allclose(O.solve(np.roll(f, 5, axis=2), g), np.roll(O.solve(f, g), 5, axis=2), atol=1e-12)


def test_helmholtz_small_alpha_returns_rhs():
    g = make_grid(8, 8, 8, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_D, O.BC_D))
    f = RNG.standard_normal((8, 8, 8))
    assert O.rel_l2(O.solve(f, g, 1e-12), f) < 1e-9


@pytest.mark.parametrize("zlo,zhi", [(O.BC_N, O.BC_N), (O.BC_D, O.BC_D), (O.BC_D, O.BC_N), (O.BC_N, O.BC_D),
                                     (O.BC_DF, O.BC_DF)])
@pytest.mark.parametrize("alpha", [1e-4, 2e-2])
def test_z_line_solves_against_stencil_and_full_method(zlo, zhi, alpha):
    """Eq. 21 (implicit along z only): every line's stencil residual, through
    apply_M on a 1 x 1 x nz grid, vanishes; and the full expansion method on a
    single line (one mode, lambda = 0) gives the same line."""
    nz = 23
    g = make_grid(3, 2, nz, (O.BC_P, O.BC_P, O.BC_N, O.BC_N, zlo, zhi), beta=1.6)
    f = RNG.standard_normal((nz, 2, 3))
    u = O.solve_z_lines(f, g, alpha)
    g1 = O.Grid(1, 1, nz, g.dx, g.dy, g.dzc, g.dzf, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, zlo, zhi))
    for j in range(2):
        for i in range(3):
            line = u[:, j, i].reshape(nz, 1, 1)
            fl = f[:, j, i].reshape(nz, 1, 1)
            assert np.allclose(O.apply_M(line, g1, alpha), fl, atol=1e-12)
            assert O.rel_l2(O.solve(fl, g1, alpha), line) <= 1e-13


def test_z_line_solve_small_alpha_returns_rhs():
    g = make_grid(4, 3, 16, (O.BC_N, O.BC_N, O.BC_D, O.BC_D, O.BC_D, O.BC_N))
    f = RNG.standard_normal((16, 3, 4))
    assert O.rel_l2(O.solve_z_lines(f, g, 1e-12), f) < 1e-9


def test_staggered_div_grad_is_laplacian_and_projection():
    g = make_grid(8, 6, 10, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_N, O.BC_N), beta=1.8)
    phi = RNG.standard_normal((10, 6, 8))
    assert np.allclose(O.divergence(*O.gradient(phi, g), g), O.apply_L(phi, g), atol=1e-9)
    u, v, w = S.velocity_field(3, 8, 6, 10)
    d = O.divergence(u, v, w, g)
    assert abs((d * g.dzf.reshape(-1, 1, 1)).sum()) < 1e-10       # consistent RHS (R9)
    pu = O.project_velocity([u, v, w], g)
    assert np.abs(O.divergence(*pu, g)).max() < 1e-10 * np.abs(d).max()
    assert all(np.allclose(a, b, atol=1e-10) for a, b in zip(O.project_velocity(pu, g), pu))


def test_div_grad_transposes():
    g = make_grid(5, 4, 6, (O.BC_P, O.BC_P, O.BC_P, O.BC_P, O.BC_N, O.BC_N))
    u, v, w = RNG.standard_normal((3, 6, 4, 5))
    w = np.concatenate([np.zeros((1, 4, 5)), RNG.standard_normal((5, 4, 5)), np.zeros((1, 4, 5))])
    d = RNG.standard_normal((6, 4, 5))
    dt = O.divergence_T(d, g)
    lhs = (O.divergence(u, v, w, g) * d).sum()
    rhs = (u * dt[0]).sum() + (v * dt[1]).sum() + (w * dt[2]).sum()
    assert np.isclose(lhs, rhs, rtol=1e-12)
    gx, gy, gz = O.gradient(d, g)
    a, b = RNG.standard_normal((2, 6, 4, 5))
    c = np.concatenate([np.zeros((1, 4, 5)), RNG.standard_normal((5, 4, 5)), np.zeros((1, 4, 5))])
    lhs = (gx * a).sum() + (gy * b).sum() + (gz * c).sum()
    assert np.isclose(lhs, (d * O.gradient_T(a, b, c, g)).sum(), rtol=1e-12)


def test_rk3_coefficients_fixture():
    rows = [ln.split() for ln in (Path(__file__).parent / "golden" / "rk3_coefficients.txt").read_text().splitlines()
            if ln.strip() and not ln.startswith("#")]
    alpha = [Fraction(r[1]) for r in rows]
    beta = [Fraction(r[2]) for r in rows]
    gamma = [a + b for a, b in zip(alpha, beta)]
    assert gamma == [Fraction(8, 15), Fraction(2, 15), Fraction(1, 3)]
    assert sum(gamma) == 1          # the three substeps advance one full time step


# ---------------------------------------------------------------------------
# mutation tests: plausible mistakes planted in the oracle must fail a pin
# ---------------------------------------------------------------------------
def _dense_mismatch(g, alpha=None):
    f = RNG.standard_normal((g.nz, g.ny, g.nx))
    return O.rel_l2(O.solve(f, g, alpha), O.dense_solve(f, g, alpha))


def test_mutation_eigenvalue_sign_is_caught(monkeypatch):
    orig = O.cales_oracle.eigenvalues
    monkeypatch.setattr(O.cales_oracle, "eigenvalues", lambda k, n, h: -orig(k, n, h))
    assert _dense_mismatch(make_grid(6, 4, 5, (0, 0, 1, 1, 1, 1))) > 1e-3


def test_mutation_transposed_z_operator_is_caught(monkeypatch):
    orig = O.cales_oracle.z_operator

    def swapped(g):
        sub, diag, sup = orig(g)
        s2 = np.zeros_like(sub)
        s2[1:] = sup[:-1]
        u2 = np.zeros_like(sup)
        u2[:-1] = sub[1:]
        return s2, diag, u2
    monkeypatch.setattr(O.cales_oracle, "z_operator", swapped)
    assert _dense_mismatch(make_grid(4, 4, 9, (0, 0, 0, 0, 2, 1), beta=2.0)) > 1e-6


def test_mutation_dropped_neumann_ghost_is_caught(monkeypatch):
    orig = O.cales_oracle.z_operator

    def dropped(g):
        sub, diag, sup = orig(g)
        diag = diag.copy()
        diag[0] -= 1.0 / (g.dzc[0] * g.dzf[0])
        return sub, diag, sup
    monkeypatch.setattr(O.cales_oracle, "z_operator", dropped)
    assert _dense_mismatch(make_grid(4, 4, 6, (0, 0, 0, 0, 1, 1)), alpha=1e-2) > 1e-6


def test_mutation_spacing_swap_fails_convergence():
    """Swapping the roles of dzc and dzf leaves only first-order convergence."""
    errs = []
    for nz in (32, 64, 128):
        zf = S.tanh_faces(nz, 1.8)
        dzc, dzf = O.cell_spacings(zf)
        g = O.Grid(1, 1, nz, 1.0, 1.0, dzf.tolist() + [dzf[-1]], dzc[:-1], (0, 0, 0, 0, 1, 1))
        zc = 0.5 * (zf[1:] + zf[:-1])
        p = np.cos(math.pi * zc).reshape(-1, 1, 1)
        inner = slice(nz // 4, 3 * nz // 4)
        errs.append(np.abs((O.apply_L(p, g) + math.pi ** 2 * p)[inner]).max())
    assert errs[0] / errs[1] < 3.2 or errs[1] / errs[2] < 3.2
