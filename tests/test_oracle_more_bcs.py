"""Pins of the oracle's transforms for face-centred unknowns (DST-I) and mixed
Neumann / Dirichlet sides (DCT-IV, DST-IV) in the uniform directions:
library transforms, discrete eigenfunctions of the ghost rules, dense LU of
the whole operator, and a planted mistake."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.cales_oracle as C
import synth_inputs as S

scipy_fft = pytest.importorskip("scipy.fft")


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_transforms_match_library(n):
    x = S.gaussian(600 + n, (n,))
    assert np.allclose(2 * O.fwd_matrix(O.BC_DF, n) @ x, scipy_fft.dst(x, type=1), atol=1e-12)
    assert np.allclose(2 * O.fwd_matrix(O.KIND_ND, n) @ x, scipy_fft.dct(x, type=4), atol=1e-12)
    assert np.allclose(2 * O.fwd_matrix(O.KIND_DN, n) @ x, scipy_fft.dst(x, type=4), atol=1e-12)
    for kind in (O.BC_DF, O.KIND_ND, O.KIND_DN):
        assert np.allclose(O.inv_matrix(kind, n) @ O.fwd_matrix(kind, n), np.eye(n), atol=1e-12)


@pytest.mark.parametrize("lo,hi", [(O.BC_DF, O.BC_DF), (O.BC_N, O.BC_D), (O.BC_D, O.BC_N)])
@pytest.mark.parametrize("n", [3, 8])
def test_basis_vectors_are_eigenvectors_of_the_ghost_rules(lo, hi, n):
    """Each row of the forward matrix is an eigenvector of the 1-D second
    difference with the sides' ghosts (DF: zero at the boundary node; N: the
    ghost repeats the first value; D: minus it), with the printed eigenvalue."""
    h = 0.3
    g = O.Grid(n, 1, 3, h, 1.0, np.ones(4), np.ones(3), (lo, hi, O.BC_P, O.BC_P, O.BC_N, O.BC_N))
    kind = O.dir_kind(lo, hi)
    lam = O.eigenvalues(kind, n, h)
    basis = O.fwd_matrix(kind, n)
    for m in range(n):
        v = np.broadcast_to(basis[m][None, None, :], (3, 1, n)).copy()
        lv = O.apply_L(v, g)
        assert np.max(np.abs(lv - lam[m] * v)) <= 1e-12 * (abs(lam[m]) + 1.0 / h ** 2)


@pytest.mark.parametrize("bcx", [(O.BC_DF, O.BC_DF), (O.BC_N, O.BC_D), (O.BC_D, O.BC_N), (O.BC_P, O.BC_P)])
@pytest.mark.parametrize("bcy", [(O.BC_N, O.BC_D), (O.BC_DF, O.BC_DF), (O.BC_N, O.BC_N)])
@pytest.mark.parametrize("alpha", [None, 0.02])
def test_solve_matches_dense_lu(bcx, bcy, alpha):
    zf = S.tanh_faces(5, 1.6, 2.0)
    dzc, dzf = O.cell_spacings(zf)
    nx = 4 if bcx[0] == O.BC_P else 5
    g = O.Grid(nx, 3, 5, 0.4, 0.7, dzc, dzf, bcx + bcy + (O.BC_N, O.BC_D))
    f = S.gaussian(650 + nx + bcy[0], (5, 3, nx))
    assert O.rel_l2(O.solve(f, g, alpha), O.dense_solve(f, g, alpha)) < 1e-11


def test_mixed_sides_without_dirichlet_are_not_singular_unless_all_neumann():
    zf = S.tanh_faces(4, 1.2, 2.0)
    dzc, dzf = O.cell_spacings(zf)
    g = O.Grid(4, 4, 4, 0.5, 0.5, dzc, dzf, (O.BC_N, O.BC_D, O.BC_N, O.BC_N, O.BC_N, O.BC_N))
    assert not O.is_singular(g)
    g2 = O.Grid(4, 4, 4, 0.5, 0.5, dzc, dzf, (O.BC_N, O.BC_N, O.BC_P, O.BC_P, O.BC_N, O.BC_N))
    assert O.is_singular(g2)


def test_mutation_swapped_mixed_transforms_fail_the_dense_pin(monkeypatch):
    real = C.dir_kind
    swap = {O.KIND_ND: O.KIND_DN, O.KIND_DN: O.KIND_ND}
    monkeypatch.setattr(C, "dir_kind", lambda lo, hi: swap.get(real(lo, hi), real(lo, hi)))
    with pytest.raises(AssertionError):
        test_solve_matches_dense_lu((O.BC_N, O.BC_D), (O.BC_N, O.BC_N), 0.02)
