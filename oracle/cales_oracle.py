"""Plain FP64 oracle of the eigenfunction-expansion fast direct solver.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
uses this module.

What it computes.  The paper (Sec. 2.2) discretises the Poisson equation for
the pressure correction, Eq. (12), and the Crank-Nicolson velocity Helmholtz
equations, Eq. (18), with second-order finite differences on a staggered
(MAC) grid and solves both with the same direct method: an eigenfunction
expansion (Schumann & Sweet) in the two uniform directions and the Thomas
algorithm along the non-uniform direction z (the paper's text calls the
wall-normal direction "y" but the solver stretches z).

The discrete operator is not printed in the paper.  Readings used here:

R1  L p = (p[i+1]-2p[i]+p[i-1])/dx^2 + (p[j+1]-2p[j]+p[j-1])/dy^2
        + ((p[k+1]-p[k])/dzc[k+1] - (p[k]-p[k-1])/dzc[k]) / dzf[k]
R2  ghost values: periodic wraps; N (zero flux at the face): p[-1] = p[0];
    D (zero value at the face, cell-centred unknown): p[-1] = -p[0] with the
    mirror spacing dzc[0]; DF (zero value at a boundary node, node-centred
    unknown): p[-1] = 0 at distance dzc[0].
R3  Poisson with no Dirichlet side is singular: the right-hand side is made
    consistent by subtracting its dzf-weighted mean (sum dzf * L p == 0).
R4  the zero mode is pinned by replacing its last row with p_hat = 0.
R5  the result is gauged to zero dzf-weighted mean.

Every transform is an explicit O(n^2) matrix (complex DFT for periodic
directions, DCT-II for Neumann, DST-II for Dirichlet); the tridiagonal
systems are solved by scalar Thomas elimination (vectorised over modes, the
recurrence itself runs index by index).  Numpy's matmul is the only library
primitive on the solve path.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_P, BC_N, BC_D, BC_DF = 0, 1, 2, 3
BC_NAMES = {"P": BC_P, "N": BC_N, "D": BC_D, "DF": BC_DF}

__all__ = [
    "BC_P", "BC_N", "BC_D", "BC_DF", "BC_NAMES", "KIND_ND", "KIND_DN", "dir_kind", "Grid", "cell_spacings",
    "face_spacings", "apply_L", "apply_M", "fwd_matrix", "inv_matrix",
    "eigenvalues", "z_operator", "thomas", "is_singular", "weighted_mean",
    "project", "solve", "solve_refined", "solve_z_lines", "solve_T", "dense_matrix", "dense_solve", "residual",
    "rel_l2", "divergence", "gradient", "divergence_T", "gradient_T",
]


# ---------------------------------------------------------------------------
# Grid
# ---------------------------------------------------------------------------
@dataclass
class Grid:
    """Staggered grid: uniform dx, dy; z spacings dzc[0..nz] and dzf[0..nz-1].

    dzf[k] is the width of the control volume of unknown k, dzc[k] the
    distance between unknowns k-1 and k (dzc[0], dzc[nz]: distance to the
    ghost / boundary node).  bc = (xlo, xhi, ylo, yhi, zlo, zhi).
    """

    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dzc: np.ndarray
    dzf: np.ndarray
    bc: tuple = (BC_P, BC_P, BC_P, BC_P, BC_N, BC_N)
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        self.dzc = np.asarray(self.dzc, dtype=np.float64)
        self.dzf = np.asarray(self.dzf, dtype=np.float64)
        assert self.dzc.shape == (self.nz + 1,) and self.dzf.shape == (self.nz,)
        self.bc = tuple(int(b) for b in self.bc)


def cell_spacings(zf: np.ndarray):
    """dzc, dzf of cell-centred unknowns from the faces zf[0..nz] (mirror ends)."""
    zf = np.asarray(zf, dtype=np.float64)
    dzf = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzc = np.empty(len(zf))
    dzc[1:-1] = np.diff(zc)
    dzc[0] = dzf[0]
    dzc[-1] = dzf[-1]
    return dzc, dzf


def face_spacings(zf: np.ndarray):
    """dzc, dzf of node-centred unknowns on the interior faces zf[1..nz-1].

    The unknowns sit on faces; their control volumes span neighbouring cell
    centres, and the boundary nodes zf[0], zf[nz] carry the Dirichlet value.
    """
    zf = np.asarray(zf, dtype=np.float64)
    dz_cells = np.diff(zf)                    # distance between consecutive nodes
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzf_w = np.diff(zc)                       # control volume of face k+1, k=0..nz-2
    return dz_cells.copy(), dzf_w


# ---------------------------------------------------------------------------
# Discrete operator (readings R1, R2)
# ---------------------------------------------------------------------------
def _neighbours(p: np.ndarray, axis: int, lo: int, hi: int):
    """(p[i-1], p[i+1]) along ``axis`` with the R2 ghost values."""
    n = p.shape[axis]
    if lo == BC_P:
        return np.roll(p, 1, axis=axis), np.roll(p, -1, axis=axis)
    first = np.take(p, [0], axis=axis)
    last = np.take(p, [n - 1], axis=axis)
    gl = {BC_N: first, BC_D: -first, BC_DF: 0.0 * first}[lo]
    gh = {BC_N: last, BC_D: -last, BC_DF: 0.0 * last}[hi]
    lower = np.concatenate([gl, np.take(p, np.arange(0, n - 1), axis=axis)], axis=axis)
    upper = np.concatenate([np.take(p, np.arange(1, n), axis=axis), gh], axis=axis)
    return lower, upper


def apply_L(p: np.ndarray, g: Grid) -> np.ndarray:
    """Staggered 7-point Laplacian of Eq. (16) (readings R1, R2); p is [nz][ny][nx]."""
    xm, xp = _neighbours(p, 2, g.bc[0], g.bc[1])
    ym, yp = _neighbours(p, 1, g.bc[2], g.bc[3])
    zm, zp = _neighbours(p, 0, g.bc[4], g.bc[5])
    out = (xp - 2.0 * p + xm) / g.dx ** 2 + (yp - 2.0 * p + ym) / g.dy ** 2
    dzc = g.dzc.reshape(-1, 1, 1)
    dzf = g.dzf.reshape(-1, 1, 1)
    out = out + ((zp - p) / dzc[1:] - (p - zm) / dzc[:-1]) / dzf
    return out


def apply_M(p: np.ndarray, g: Grid, alpha=None) -> np.ndarray:
    """L p for Poisson (alpha None), (I - alpha L) p for the Helmholtz form of Eq. (18)."""
    lp = apply_L(p, g)
    return lp if alpha is None else p - alpha * lp


def residual(p, f, g: Grid, alpha=None):
    return f - apply_M(p, g, alpha)


# ---------------------------------------------------------------------------
# Transforms of the uniform directions (explicit matrices) and eigenvalues
# ---------------------------------------------------------------------------
def _cos_sin_frac(num: np.ndarray, den: int):
    """cos and sin of 2*pi*num/den with the integer argument reduced exactly."""
    r = np.mod(num, den).astype(np.float64) / den
    return np.cos(2.0 * math.pi * r), np.sin(2.0 * math.pi * r)


# Transform kinds of a uniform direction with different sides: Neumann below
# and Dirichlet above (KIND_ND), or the reverse (KIND_DN).
KIND_ND, KIND_DN = 4, 5


def dir_kind(lo: int, hi: int) -> int:
    """Transform kind of a uniform direction from its two sides."""
    if lo == hi:
        return lo
    if (lo, hi) == (BC_N, BC_D):
        return KIND_ND
    if (lo, hi) == (BC_D, BC_N):
        return KIND_DN
    raise ValueError(f"no transform for the sides ({lo}, {hi})")


def fwd_matrix(kind: int, n: int) -> np.ndarray:
    """Forward transform matrix of one uniform direction.

    P : F[m, i] = exp(-2 pi i m i / n)                  (complex DFT)
    N : C[m, i] = cos(pi m (i + 1/2) / n), m = 0..n-1    (DCT-II)
    D : S[m, i] = sin(pi m (i + 1/2) / n), m = 1..n      (DST-II), row m-1
    DF: S[m, i] = sin(pi (m+1) (i+1) / (n+1))            (DST-I; n interior nodes)
    ND: C[m, i] = cos(pi (m + 1/2) (i + 1/2) / n)        (DCT-IV)
    DN: S[m, i] = sin(pi (m + 1/2) (i + 1/2) / n)        (DST-IV)
    """
    i = np.arange(n, dtype=np.int64)
    if kind == BC_DF:
        _, s = _cos_sin_frac(np.outer(i + 1, i + 1), 2 * (n + 1))
        return s
    if kind in (KIND_ND, KIND_DN):
        c, s = _cos_sin_frac(np.outer(2 * i + 1, 2 * i + 1), 8 * n)
        return c if kind == KIND_ND else s
    if kind == BC_P:
        c, s = _cos_sin_frac(np.outer(i, i), n)
        return c - 1j * s
    if kind == BC_N:
        m = np.arange(n, dtype=np.int64)
        c, _ = _cos_sin_frac(np.outer(m, 2 * i + 1), 4 * n)
        return c
    if kind == BC_D:
        m = np.arange(1, n + 1, dtype=np.int64)
        _, s = _cos_sin_frac(np.outer(m, 2 * i + 1), 4 * n)
        return s
    raise ValueError(f"no transform for bc kind {kind} in a uniform direction")


def inv_matrix(kind: int, n: int) -> np.ndarray:
    """Inverse of ``fwd_matrix`` written out from the orthogonality relations.

    P : conj(F)^T / n.   N : DCT-III with weights 1/n (m=0) and 2/n.
    D : DST-III with weights 2/n (m<n) and 1/n (m=n).
    DF, ND, DN: the matrices are symmetric and orthogonal up to the factor
    (n+1)/2 resp. n/2, so the inverse is 2/(n+1) resp. 2/n times the matrix.
    """
    i = np.arange(n, dtype=np.int64)
    if kind == BC_DF:
        return fwd_matrix(BC_DF, n) * (2.0 / (n + 1))
    if kind in (KIND_ND, KIND_DN):
        return fwd_matrix(kind, n) * (2.0 / n)
    if kind == BC_P:
        return np.conj(fwd_matrix(BC_P, n)).T / n
    if kind == BC_N:
        m = np.arange(n, dtype=np.int64)
        c, _ = _cos_sin_frac(np.outer(2 * i + 1, m), 4 * n)
        w = np.full(n, 2.0 / n)
        w[0] = 1.0 / n
        return c * w[None, :]
    if kind == BC_D:
        m = np.arange(1, n + 1, dtype=np.int64)
        _, s = _cos_sin_frac(np.outer(2 * i + 1, m), 4 * n)
        w = np.full(n, 2.0 / n)
        w[-1] = 1.0 / n
        return s * w[None, :]
    raise ValueError(kind)


def eigenvalues(kind: int, n: int, h: float) -> np.ndarray:
    """Modified wavenumbers of the 3-point second difference with R2 ghosts.

    P : -(4/h^2) sin^2(pi m / n),      m = 0..n-1
    N : -(4/h^2) sin^2(pi m / (2n)),   m = 0..n-1
    D : -(4/h^2) sin^2(pi m / (2n)),   m = 1..n
    DF: -(4/h^2) sin^2(pi m / (2(n+1))), m = 1..n      (h: node spacing)
    ND, DN: -(4/h^2) sin^2(pi (2m+1) / (4n)), m = 0..n-1
    """
    if kind == BC_DF:
        m = np.arange(1, n + 1)
        return -(4.0 / h ** 2) * np.sin(math.pi * m / (2.0 * (n + 1))) ** 2
    if kind in (KIND_ND, KIND_DN):
        m = np.arange(n)
        return -(4.0 / h ** 2) * np.sin(math.pi * (2 * m + 1) / (4.0 * n)) ** 2
    if kind == BC_P:
        m = np.arange(n)
        return -(4.0 / h ** 2) * np.sin(math.pi * m / n) ** 2
    if kind == BC_N:
        m = np.arange(n)
    elif kind == BC_D:
        m = np.arange(1, n + 1)
    else:
        raise ValueError(kind)
    return -(4.0 / h ** 2) * np.sin(math.pi * m / (2.0 * n)) ** 2


# ---------------------------------------------------------------------------
# z direction: tridiagonal operator and Thomas elimination
# ---------------------------------------------------------------------------
def z_operator(g: Grid):
    """(sub, diag, sup) of L_z with the R2 boundary rows; all length nz.

    sub[k] multiplies p[k-1] (sub[0] unused), sup[k] multiplies p[k+1]
    (sup[nz-1] unused).
    """
    nz = g.nz
    a = 1.0 / (g.dzc[:-1] * g.dzf)     # coupling of row k to k-1
    c = 1.0 / (g.dzc[1:] * g.dzf)      # coupling of row k to k+1
    diag = -(a + c)
    lo, hi = g.bc[4], g.bc[5]
    if lo == BC_P:
        # periodic: sub[0] couples row 0 to row nz-1, sup[nz-1] row nz-1 to row 0
        return a.copy(), diag, c.copy()
    diag[0] += {BC_N: a[0], BC_D: -a[0], BC_DF: 0.0}[lo]
    diag[nz - 1] += {BC_N: c[nz - 1], BC_D: -c[nz - 1], BC_DF: 0.0}[hi]
    sub = a.copy()
    sub[0] = 0.0
    sup = c.copy()
    sup[nz - 1] = 0.0
    return sub, diag, sup


def thomas(sub, diag, sup, rhs):
    """Scalar Thomas elimination without pivoting (Golub & Van Loan, Alg. 4.3.x).

    sub, sup: (n,) ; diag: (n, M) or (n,) ; rhs: (n, M).  Solves each column.
    """
    n = rhs.shape[0]
    diag = np.broadcast_to(diag if np.ndim(diag) == 2 else np.asarray(diag)[:, None], rhs.shape)
    cp = np.empty(rhs.shape, dtype=np.float64)
    dp = np.empty(rhs.shape, dtype=rhs.dtype)
    den = diag[0]
    cp[0] = sup[0] / den
    dp[0] = rhs[0] / den
    for k in range(1, n):
        den = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / den
        dp[k] = (rhs[k] - sub[k] * dp[k - 1]) / den
    x = np.empty_like(dp)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def cyclic_solve(sub, diag, sup, rhs):
    """Periodic z: the cyclic tridiagonal of each column (corners sub[0] at
    (0, n-1) and sup[n-1] at (n-1, 0)) assembled densely and solved by LAPACK
    (batched gesv).  diag: (n, M) or (n,); rhs: (n, M)."""
    n, m = rhs.shape
    diag = np.broadcast_to(diag if np.ndim(diag) == 2 else np.asarray(diag)[:, None], rhs.shape)
    mat = np.zeros((m, n, n))
    k = np.arange(n)
    mat[:, k, k] = diag.T
    mat[:, k[1:], k[:-1]] = sub[1:]
    mat[:, k[:-1], k[1:]] = sup[:-1]
    mat[:, 0, n - 1] += sub[0]
    mat[:, n - 1, 0] += sup[n - 1]
    return np.linalg.solve(mat, rhs.T[:, :, None])[:, :, 0].T


def is_singular(g: Grid, alpha=None) -> bool:
    """Poisson with only periodic/Neumann sides: constants are in the null space."""
    return alpha is None and all(b in (BC_P, BC_N) for b in g.bc)


def weighted_mean(f: np.ndarray, g: Grid) -> float:
    """dzf-weighted volume mean (readings R3, R5)."""
    w = g.dzf.reshape(-1, 1, 1)
    return float((f * w).sum() / (w.sum() * g.nx * g.ny))


def project(f: np.ndarray, g: Grid) -> np.ndarray:
    return f - weighted_mean(f, g)


def _check_supported(g: Grid):
    for lo, hi in ((g.bc[0], g.bc[1]), (g.bc[2], g.bc[3])):
        if (lo == BC_P) != (hi == BC_P) or (lo == BC_DF) != (hi == BC_DF):
            raise ValueError("uniform directions take P or DF on both sides, or N / D per side")
    if (g.bc[4] == BC_P) != (g.bc[5] == BC_P):
        raise ValueError("a periodic z is periodic on both sides")
    if g.bc[4] == BC_P and g.nz < 3:
        raise ValueError("a periodic z needs at least three cells")
    if g.bc[4] not in (BC_P, BC_N, BC_D, BC_DF) or g.bc[5] not in (BC_P, BC_N, BC_D, BC_DF):
        raise ValueError("z takes P (both sides), N, D or DF at each side")


def _apply_along(mat: np.ndarray, a: np.ndarray, axis: int) -> np.ndarray:
    """out[..., m, ...] = sum_i mat[m, i] a[..., i, ...] via one matmul."""
    a = np.moveaxis(a, axis, -1)
    shp = a.shape
    flat = a.reshape(-1, shp[-1])
    if np.iscomplexobj(mat) and not np.iscomplexobj(flat):
        out = (flat @ mat.real.T) + 1j * (flat @ mat.imag.T)
    else:
        out = flat @ mat.T
    out = out.reshape(shp[:-1] + (mat.shape[0],))
    return np.moveaxis(out, -1, axis)


def _mode_tridiag(g: Grid, alpha):
    """Per-mode tridiagonal of Poisson (L_z + lambda) or Helmholtz (I - alpha(L_z + lambda))."""
    sub, diag, sup = z_operator(g)
    lam = (eigenvalues(dir_kind(g.bc[2], g.bc[3]), g.ny, g.dy)[:, None]
           + eigenvalues(dir_kind(g.bc[0], g.bc[1]), g.nx, g.dx)[None, :]).reshape(-1)
    if alpha is None:
        return sub, diag[:, None] + lam[None, :], sup
    return -alpha * sub, 1.0 - alpha * (diag[:, None] + lam[None, :]), -alpha * sup


def solve(f: np.ndarray, g: Grid, alpha=None) -> np.ndarray:
    """p with L p = f (Poisson, Eq. 12) or (I - alpha L) p = f (Helmholtz, Eq. 18).

    Steps: [project (R3)] -> forward x, y transforms -> one tridiagonal per
    (mx, my) in z, zero mode pinned (R4) -> inverse y, x -> [gauge (R5)].
    """
    _check_supported(g)
    f = np.asarray(f, dtype=np.float64)
    nx, ny, nz = g.nx, g.ny, g.nz
    sing = is_singular(g, alpha)
    if sing:
        f = project(f, g)
    fh = _apply_along(fwd_matrix(dir_kind(g.bc[0], g.bc[1]), nx), f, 2)
    fh = _apply_along(fwd_matrix(dir_kind(g.bc[2], g.bc[3]), ny), fh, 1)
    sub, diag, sup = _mode_tridiag(g, alpha)
    rhs = fh.reshape(nz, -1)
    per = g.bc[4] == BC_P
    line = (lambda a, d, c, r: cyclic_solve(a, d, c, r)) if per else thomas
    if sing:
        ph = np.empty_like(rhs)
        ph[:, 1:] = line(sub, diag[:, 1:], sup, rhs[:, 1:])
        ph[nz - 1, 0] = 0.0
        if nz > 1:
            # pinned last unknown: the wrap couplings of rows 0 and nz-2 to it drop out
            ph[:nz - 1, :1] = thomas(sub[:nz - 1], diag[:nz - 1, :1], sup[:nz - 1], rhs[:nz - 1, :1])
    else:
        ph = line(sub, diag, sup, rhs)
    ph = ph.reshape(nz, ny, nx)
    p = _apply_along(inv_matrix(dir_kind(g.bc[2], g.bc[3]), ny), ph, 1)
    p = _apply_along(inv_matrix(dir_kind(g.bc[0], g.bc[1]), nx), p, 2)
    p = np.real(p) if np.iscomplexobj(p) else p
    if sing:
        p = p - weighted_mean(p, g)
    return np.ascontiguousarray(p)


def solve_refined(f: np.ndarray, g: Grid, alpha=None, steps: int = 1) -> np.ndarray:
    """``solve`` followed by ``steps`` rounds of FP64 iterative refinement:
    r = f - M p with the R1/R2 stencil (``apply_M``), p += solve(r).

    The method's result is the exact solution of the discrete system (Sec.
    2.2).  The plain expansion reaches it only up to cond * eps on the
    near-singular modes: the scalar Thomas elimination of a strongly
    stretched z line (512 cells, tanh beta = 1.5) has condition numbers near
    3e6, and ``solve`` then differs from the exact discrete solution by about
    1e-12 (relative L2).  One refinement step returns it to the rounding floor
    of the stencil (about 1e-16).  For a singular problem f is projected first
    (R3); every correction is gauged by ``solve`` (R5).
    """
    f = np.asarray(f, dtype=np.float64)
    if is_singular(g, alpha):
        f = project(f, g)
    p = solve(f, g, alpha)
    for _ in range(steps):
        p = p + solve(f - apply_M(p, g, alpha), g, alpha)
    return p


def solve_z_lines(f: np.ndarray, g: Grid, alpha: float) -> np.ndarray:
    """u with (I - alpha L_z) u = f on every (i, j) line independently: the
    viscous term implicit along the wall-normal direction only (Eq. 21,
    Sec. 2.2; the paper's wall-normal "y" is the stretched z here).  One
    tridiagonal per line with the R2 z boundary rows, scalar Thomas; x and y
    boundary kinds play no part."""
    sub, diag, sup = z_operator(g)
    rhs = np.asarray(f, dtype=np.float64).reshape(g.nz, -1)
    line = cyclic_solve if g.bc[4] == BC_P else thomas          # periodic z: cyclic line systems
    u = line(-alpha * sub, 1.0 - alpha * diag, -alpha * sup, rhs)
    return np.ascontiguousarray(u.reshape(g.nz, g.ny, g.nx))


def solve_T(w: np.ndarray, g: Grid, alpha=None) -> np.ndarray:
    """Transpose of the linear map f -> solve(f): every step of ``solve``
    transposed and applied in reverse order (an independent route to S^T w).
    """
    _check_supported(g)
    per = g.bc[4] == BC_P
    w = np.asarray(w, dtype=np.float64)
    nx, ny, nz = g.nx, g.ny, g.nz
    sing = is_singular(g, alpha)
    mvec = (g.dzf / (g.dzf.sum() * nx * ny)).reshape(-1, 1, 1)
    if sing:   # gauge Z = I - 1 m^T  ->  Z^T w = w - m * sum(w)
        w = w - mvec * w.sum()
    a = _apply_along(inv_matrix(dir_kind(g.bc[0], g.bc[1]), nx).T, w, 2)
    a = _apply_along(inv_matrix(dir_kind(g.bc[2], g.bc[3]), ny).T, a, 1)
    sub, diag, sup = _mode_tridiag(g, alpha)
    rhs = a.reshape(nz, -1)
    # transposed tridiagonal: sub'[k] = sup[k-1], sup'[k] = sub[k+1]; a
    # periodic z also swaps the corners: sub'[0] = sup[nz-1], sup'[nz-1] = sub[0]
    subT = np.zeros(nz)
    supT = np.zeros(nz)
    subT[1:] = sup[:-1]
    supT[:-1] = sub[1:]
    if per:
        subT[0] = sup[nz - 1]
        supT[nz - 1] = sub[0]
    if sing:
        out = np.empty_like(rhs)
        out[:, 1:] = (cyclic_solve if per else thomas)(subT, diag[:, 1:], supT, rhs[:, 1:])
        # zero mode: map g -> T_pin^{-1} diag(1,..,1,0) g; its transpose is
        # diag(1,..,1,0) T_pin^{-T} g with T_pin = rows 0..nz-2 of T plus e_last.
        tp = np.zeros((nz, nz))
        for k in range(nz - 1):
            tp[k, k] = diag[k, 0]
            if k > 0:
                tp[k, k - 1] = sub[k]
            tp[k, k + 1] = sup[k]
        tp[nz - 1, nz - 1] = 1.0
        z0 = np.linalg.solve(tp.T, rhs[:, 0])
        z0[nz - 1] = 0.0
        out[:, 0] = z0
    else:
        out = (cyclic_solve if per else thomas)(subT, diag, supT, rhs)
    out = out.reshape(nz, ny, nx)
    out = _apply_along(fwd_matrix(dir_kind(g.bc[2], g.bc[3]), ny).T, out, 1)
    out = _apply_along(fwd_matrix(dir_kind(g.bc[0], g.bc[1]), nx).T, out, 2)
    out = np.real(out) if np.iscomplexobj(out) else out
    if sing:   # projection Pi = I - 1 m^T  ->  Pi^T v = v - m * sum(v)
        out = out - mvec * out.sum()
    return np.ascontiguousarray(out)


# ---------------------------------------------------------------------------
# Dense reference (pins)
# ---------------------------------------------------------------------------
def dense_matrix(g: Grid, alpha=None) -> np.ndarray:
    """The operator as an N x N matrix: column q is M applied to unit vector q."""
    n = g.nx * g.ny * g.nz
    mat = np.empty((n, n))
    e = np.zeros(n)
    for q in range(n):
        e[q] = 1.0
        mat[:, q] = apply_M(e.reshape(g.nz, g.ny, g.nx), g, alpha).reshape(-1)
        e[q] = 0.0
    return mat


def dense_solve(f: np.ndarray, g: Grid, alpha=None) -> np.ndarray:
    """LU (LAPACK gesv, partial pivoting) on the dense operator.

    Singular case: bordered system [[L, 1], [m^T, 0]] [p; mu] = [f; 0] with
    m = dzf weights, so L p = f - mu (R3) and sum(dzf p) = 0 (R5).
    """
    mat = dense_matrix(g, alpha)
    n = mat.shape[0]
    rhs = np.asarray(f, dtype=np.float64).reshape(-1)
    if is_singular(g, alpha):
        wts = np.broadcast_to(g.dzf.reshape(-1, 1, 1), (g.nz, g.ny, g.nx)).reshape(-1)
        big = np.zeros((n + 1, n + 1))
        big[:n, :n] = mat
        big[:n, n] = 1.0
        big[n, :n] = wts
        sol = np.linalg.solve(big, np.concatenate([rhs, [0.0]]))
        return sol[:n].reshape(g.nz, g.ny, g.nx)
    return np.linalg.solve(mat, rhs).reshape(g.nz, g.ny, g.nx)


def rel_l2(a, b) -> float:
    """Relative L2 error ||a - b|| / ||b|| (reading R10)."""
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.reshape(-1))
    return float(np.linalg.norm((np.asarray(a, dtype=np.float64) - b).reshape(-1)) / (den if den > 0 else 1.0))


# ---------------------------------------------------------------------------
# Staggered divergence / gradient (right-hand side of Eq. 12, correction Eq. 13)
# ---------------------------------------------------------------------------
def divergence(u, v, w, g: Grid):
    """Cell-centred divergence of a staggered velocity (reading R9).

    u[k,j,i] sits on the x-face i+1/2, v on the y-face j+1/2 (both periodic
    here), w[k] (k = 0..nz) on z-face k with w[0] = w[nz] = 0 at the walls.
    """
    du = (u - np.roll(u, 1, axis=2)) / g.dx
    dv = (v - np.roll(v, 1, axis=1)) / g.dy
    dw = (w[1:] - w[:-1]) / g.dzf.reshape(-1, 1, 1)
    return du + dv + dw


def gradient(phi, g: Grid):
    """Face gradient of a cell-centred scalar: (gx at x-faces, gy, gz at z-faces).

    gz[0] = gz[nz] = 0 (walls, no flux correction of the wall-normal velocity).
    """
    gx = (np.roll(phi, -1, axis=2) - phi) / g.dx
    gy = (np.roll(phi, -1, axis=1) - phi) / g.dy
    gz = np.zeros((g.nz + 1,) + phi.shape[1:])
    gz[1:-1] = (phi[1:] - phi[:-1]) / g.dzc[1:-1].reshape(-1, 1, 1)
    return gx, gy, gz


def divergence_T(d, g: Grid):
    """Transpose of ``divergence`` (w's wall rows are fixed inputs -> zero)."""
    ux = (d - np.roll(d, -1, axis=2)) / g.dx
    vy = (d - np.roll(d, -1, axis=1)) / g.dy
    dd = d / g.dzf.reshape(-1, 1, 1)
    wz = np.zeros((g.nz + 1,) + d.shape[1:])
    wz[1:-1] = dd[:-1] - dd[1:]
    return ux, vy, wz


def gradient_T(gx, gy, gz, g: Grid):
    """Transpose of ``gradient``."""
    out = (np.roll(gx, 1, axis=2) - gx) / g.dx + (np.roll(gy, 1, axis=1) - gy) / g.dy
    t = gz[1:-1] / g.dzc[1:-1].reshape(-1, 1, 1)
    out = out.copy()
    out[1:] += t
    out[:-1] -= t
    return out
