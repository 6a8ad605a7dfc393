"""Pins of the RK3 pressure-correction substep oracle (Sec. 2.2, Eqs. 11-15)
against what the mathematics fixes: conservation of the divergence-form
advection, closed-form eigenfunctions of the viscous operator, the identity
d(2 c S_ij)/dx_j = c L u_i for divergence-free fields, the 1-D conservative
diffusion operator, the RK3 stability polynomial, and a divergence-free
result.  Mutations planted in the oracle fail them."""
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle as O
import oracle.rk3_oracle as R
import synth_inputs as S


def _grid(nx, ny, nz, beta, lz=2.0):
    zf = S.tanh_faces(nz, beta, lz) if beta > 0 else np.linspace(0.0, lz, nz + 1)
    dzc, dzf = O.cell_spacings(zf)
    return O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, dzc, dzf, (0, 0, 0, 0, 1, 1))


def _velocity(seed, g, divfree=True):
    u = S.gaussian(seed, (g.nz, g.ny, g.nx))
    v = S.gaussian(seed + 1, (g.nz, g.ny, g.nx))
    w = S.gaussian(seed + 2, (g.nz + 1, g.ny, g.nx))
    w[0] = 0.0
    w[-1] = 0.0
    if divfree:
        u, v, w = O.project_velocity([u, v, w], g)
    return u, v, w


def _vol(g):
    return (g.dx * g.dy * g.dzf).reshape(-1, 1, 1), (g.dx * g.dy * g.dzc[1:-1]).reshape(-1, 1, 1)


def test_coefficients_are_the_printed_fractions():
    rows = [ln.split() for ln in (Path(__file__).parent / "golden" / "rk3_coefficients.txt").read_text().splitlines()
            if ln.strip() and not ln.startswith("#")]
    for k, r in enumerate(rows):
        assert O.RK3_ALPHA[k] == float(Fraction(r[1])) and O.RK3_BETA[k] == float(Fraction(r[2]))
    assert abs(sum(O.RK3_GAMMA) - 1.0) < 1e-15


def test_advection_conserves_momentum():
    g = _grid(12, 10, 9, 1.7)
    u, v, w = _velocity(31, g, divfree=False)
    au, av, _ = O.advection(u, v, w, g)
    vc, _ = _vol(g)
    scale = np.sum(np.abs(au) * vc)
    assert abs(np.sum(au * vc)) <= 1e-13 * scale
    assert abs(np.sum(av * vc)) <= 1e-13 * scale


def test_advection_conserves_energy_for_divergence_free_fields():
    """Uniform staggered grid: the divergence form with mean interpolation
    does no work on a discretely divergence-free field (Morinishi et al.)."""
    g = _grid(12, 10, 8, 0.0)
    u, v, w = _velocity(41, g)
    assert np.max(np.abs(O.divergence(u, v, w, g))) < 1e-11
    au, av, aw = O.advection(u, v, w, g)
    vc, vf = _vol(g)
    terms = [u * au * vc, v * av * vc, w[1:-1] * aw[1:-1] * vf]
    total = sum(np.sum(t) for t in terms)
    scale = sum(np.sum(np.abs(t)) for t in terms)
    assert abs(total) <= 1e-12 * scale
    # and it does work on a field that is not divergence-free
    u2, v2, w2 = _velocity(41, g, divfree=False)
    a2 = O.advection(u2, v2, w2, g)
    work = np.sum(u2 * a2[0] * vc) + np.sum(v2 * a2[1] * vc) + np.sum(w2[1:-1] * a2[2][1:-1] * vf)
    assert abs(work) > 1e-3 * sum(np.sum(np.abs(t)) for t in (u2 * a2[0] * vc, v2 * a2[1] * vc))


@pytest.mark.parametrize("mx,my,mz", [(1, 2, 1), (3, 1, 2), (0, 0, 3)])
def test_viscous_operator_eigenfunctions(mx, my, mz):
    nx, ny, nz = 16, 12, 10
    g = _grid(nx, ny, nz, 0.0)
    dz = g.dzf[0]
    i, j = np.arange(nx), np.arange(ny)
    kc, kf = np.arange(nz) + 0.5, np.arange(nz + 1)
    xy = np.cos(2 * np.pi * mx * i / nx)[None, None, :] * np.cos(2 * np.pi * my * j / ny)[None, :, None]
    u = np.sin(np.pi * mz * kc / nz)[:, None, None] * xy
    w = np.sin(np.pi * mz * kf / nz)[:, None, None] * xy
    lam = (-4 / g.dx ** 2 * np.sin(np.pi * mx / nx) ** 2 - 4 / g.dy ** 2 * np.sin(np.pi * my / ny) ** 2
           - 4 / dz ** 2 * np.sin(np.pi * mz / (2 * nz)) ** 2)
    lu, lv, lw = O.viscous(u, u, w, g)
    assert np.max(np.abs(lu - lam * u)) <= 1e-11 * abs(lam)
    assert np.max(np.abs(lv - lam * u)) <= 1e-11 * abs(lam)
    assert np.max(np.abs(lw - lam * w)) <= 1e-11 * abs(lam)


def test_viscous_matches_the_dirichlet_poisson_stencil_on_stretched_grids():
    """u and v take the cell-centred Dirichlet ghost of the solver's stencil."""
    g = _grid(10, 8, 11, 1.9)
    u, v, w = _velocity(51, g, divfree=False)
    gd = O.Grid(g.nx, g.ny, g.nz, g.dx, g.dy, g.dzc, g.dzf, (0, 0, 0, 0, O.BC_D, O.BC_D))
    lu, lv, _ = O.viscous(u, v, w, g)
    assert O.rel_l2(lu, O.apply_L(u, gd)) < 1e-13
    assert O.rel_l2(lv, O.apply_L(v, gd)) < 1e-13


def test_sgs_with_constant_viscosity_is_viscous_for_divergence_free_fields():
    """d(2 c S_ij)/dx_j = c (L u_i + d_i div u) = c L u_i, walls included."""
    g = _grid(12, 10, 9, 1.8)
    u, v, w = _velocity(61, g)
    c = 0.37
    nut = np.full((g.nz, g.ny, g.nx), c)
    d = O.sgs_divergence(u, v, w, nut, g)
    lap = O.viscous(u, v, w, g)
    for a, b in zip(d, lap):
        assert O.rel_l2(a, c * b) < 1e-11


def test_sgs_of_a_wall_normal_shear_is_conservative_diffusion():
    """u = u(z), v = w = 0, nu_t = nu_t(z): the x-momentum SGS term reduces to
    the 1-D flux form [nf (du/dz)]_{k+1} - [...]_k over dzf_k, nf the mean
    of the two centres (T4 ghost copy), u ghosts minus the first value."""
    g = _grid(6, 4, 9, 1.6)
    prof = S.gaussian(71, (g.nz,))
    nprof = S.uniform(72, (g.nz,), 0.1, 1.0)
    u = np.broadcast_to(prof[:, None, None], (g.nz, g.ny, g.nx)).copy()
    nut = np.broadcast_to(nprof[:, None, None], (g.nz, g.ny, g.nx)).copy()
    zero = np.zeros_like(u)
    du, dv, dw = O.sgs_divergence(u, zero, np.zeros((g.nz + 1, g.ny, g.nx)), nut, g)
    ref = np.empty(g.nz)
    for k in range(g.nz):
        um = prof[k - 1] if k > 0 else -prof[0]
        up = prof[k + 1] if k < g.nz - 1 else -prof[-1]
        nm = 0.5 * (nprof[k - 1] + nprof[k]) if k > 0 else nprof[0]
        nq = 0.5 * (nprof[k] + nprof[k + 1]) if k < g.nz - 1 else nprof[-1]
        ref[k] = (nq * (up - prof[k]) / g.dzc[k + 1] - nm * (prof[k] - um) / g.dzc[k]) / g.dzf[k]
    assert np.max(np.abs(du - ref[:, None, None])) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(dv)) == 0.0 and np.max(np.abs(dw)) == 0.0


def _shear_mode_step(g, m, nu, dt):
    kc = np.arange(g.nz) + 0.5
    u = np.broadcast_to(np.sin(np.pi * m * kc / g.nz)[:, None, None], (g.nz, g.ny, g.nx)).copy()
    v = np.zeros_like(u)
    w = np.zeros((g.nz + 1, g.ny, g.nx))
    p = np.zeros_like(u)
    nut = np.zeros_like(u)
    r = None
    u0 = u.copy()
    for s in range(3):
        u, v, w, p, nut, r = O.rk3_substep(u, v, w, p, nut, r, g, s, dt, nu, 0.0, 1.0)
    return u0, u, v, w, p


def test_rk3_amplification_of_a_decaying_shear_mode():
    """A wall-normal shear mode is an eigenfunction of nu L with no advection
    and no pressure: one full step multiplies it by 1 + z + z^2/2 + z^3/6,
    z = nu lambda dt (three-stage, third-order Runge-Kutta)."""
    g = _grid(8, 6, 12, 0.0)
    m, nu, dt = 3, 0.02, 0.05
    u0, u, v, w, p = _shear_mode_step(g, m, nu, dt)
    lam = -4 / g.dzf[0] ** 2 * np.sin(np.pi * m / (2 * g.nz)) ** 2
    z = nu * lam * dt
    amp = 1 + z + z * z / 2 + z ** 3 / 6
    assert np.max(np.abs(u - amp * u0)) <= 1e-13
    assert np.max(np.abs(v)) == 0.0 and np.max(np.abs(w)) <= 1e-15 and np.max(np.abs(p)) <= 1e-12


def test_substep_result_is_divergence_free_and_pressure_consistent():
    g = _grid(12, 8, 10, 1.8)
    u, v, w = _velocity(81, g, divfree=False)
    p = S.gaussian(84, (g.nz, g.ny, g.nx))
    nut = O.eddy_viscosity(u, v, w, g, 0.1, 1e-3, 0.05)
    r = r_prev = None
    for s in range(3):
        dt = 1e-3
        un, vn, wn, pn, nutn, r = O.rk3_substep(u, v, w, p, nut, r, g, s, dt, 1e-3, 0.1, 0.05)
        scale = np.max(np.abs(O.divergence(u, v, w, g))) + 1.0
        assert np.max(np.abs(O.divergence(un, vn, wn, g))) <= 1e-10 * scale
        assert np.max(np.abs(wn[0])) == 0.0 and np.max(np.abs(wn[-1])) == 0.0
        # the velocity correction is -grad of gamma dt (p^{k+1/2} - p^{k-1/2}) (Eqs. 13-14)
        gm = O.RK3_GAMMA[s]
        a = O.momentum_rhs(u, v, w, nut, g, 1e-3)
        gp = O.gradient(p, g)
        gphi = O.gradient((pn - p) * gm * dt, g)
        for c, cn, ac, rp, gc, gf in zip((u, v, w), (un, vn, wn), a, r_prev or (0, 0, 0), gp, gphi):
            star = c + dt * (O.RK3_ALPHA[s] * ac + O.RK3_BETA[s] * rp - gm * gc)
            assert np.max(np.abs((star - gf)[1:-1] - cn[1:-1])) <= 1e-10 * (np.max(np.abs(cn)) + 1.0)
        r_prev = r
        assert O.rel_l2(nutn, O.eddy_viscosity(un, vn, wn, g, 0.1, 1e-3, 0.05)) == 0.0
        u, v, w, p, nut = un, vn, wn, pn, nutn


# ---------------------------------------------------------------------------
# mutations planted in the oracle fail a pin
# ---------------------------------------------------------------------------
def test_mutation_wrong_beta_fails_the_amplification_pin(monkeypatch):
    monkeypatch.setattr(R, "RK3_BETA", (0.0, -17.0 / 60.0, -5.0 / 12.0 + 0.01))
    with pytest.raises(AssertionError):
        test_rk3_amplification_of_a_decaying_shear_mode()


def test_mutation_neumann_ghost_fails_the_eigenfunction_pin(monkeypatch):
    real = R._ghost
    monkeypatch.setattr(R, "_ghost", lambda c, sign: real(c, abs(sign)))
    with pytest.raises(AssertionError):
        test_viscous_operator_eigenfunctions(1, 2, 1)


def test_mutation_west_neighbour_fails_the_energy_pin(monkeypatch):
    real = R._x
    monkeypatch.setattr(R, "_x", lambda a, s: real(a, abs(s)))       # i+1 where i-1 is meant
    with pytest.raises(AssertionError):
        test_advection_conserves_energy_for_divergence_free_fields()


# ---------------------------------------------------------------------------
# Crank-Nicolson variants (Eqs. 17-19: implicit = 1; Eqs. 20-22: implicit = 2)
# ---------------------------------------------------------------------------
def test_velocity_grids_reproduce_the_viscous_operator():
    """The implicit solves' grids carry the same Laplacian as the explicit
    viscous term: u on the Dirichlet cell grid, w on the interior-face grid."""
    g = _grid(10, 8, 11, 1.9)
    u, v, w = _velocity(91, g, divfree=False)
    guv, gw = O.velocity_grids(g)
    lu, _, lw = O.viscous(u, v, w, g)
    assert O.rel_l2(lu, O.apply_L(u, guv)) < 1e-13
    assert O.rel_l2(lw[1:-1], O.apply_L(w[1:-1], gw)) < 1e-13


def _eigen_step(g, field, mx, mz, nu, dt, implicit):
    nx, nz = g.nx, g.nz
    kc = np.arange(nz) + 0.5
    x = np.cos(2 * np.pi * mx * np.arange(nx) / nx)
    mode = np.broadcast_to(np.sin(np.pi * mz * kc / nz)[:, None, None] * x[None, None, :], (nz, g.ny, nx)).copy()
    zero = np.zeros_like(mode)
    u, v = (mode, zero) if field == "u" else (zero, mode)
    w = np.zeros((nz + 1, g.ny, nx))
    p, nut, r = zero.copy(), zero.copy(), None
    for s in range(3):
        u, v, w, p, nut, r = O.rk3_substep(u, v, w, p, nut, r, g, s, dt, nu, 0.0, 1.0, implicit)
    return mode, (u if field == "u" else v), p


@pytest.mark.parametrize("implicit", [1, 2])
def test_cn_amplification_of_a_wall_normal_shear_mode(implicit):
    """u = u(z) eigenmode, no advection or pressure: each substep multiplies it
    by (1 + gamma z/2) / (1 - gamma z/2), z = nu lambda dt."""
    g = _grid(8, 6, 12, 0.0)
    nu, dt, m = 0.05, 0.2, 2
    mode, out, p = _eigen_step(g, "u", 0, m, nu, dt, implicit)
    lam = -4 / g.dzf[0] ** 2 * np.sin(np.pi * m / (2 * g.nz)) ** 2
    amp = np.prod([(1 + gm * nu * lam * dt / 2) / (1 - gm * nu * lam * dt / 2) for gm in O.RK3_GAMMA])
    assert np.max(np.abs(out - amp * mode)) <= 1e-13
    assert np.max(np.abs(p)) <= 1e-12


@pytest.mark.parametrize("implicit", [1, 2])
def test_cn_split_of_an_x_z_mode(implicit):
    """v = X(x) Z(z) (divergence-free, no advection): implicit = 1 treats the
    whole eigenvalue by Crank-Nicolson; implicit = 2 carries the x part with
    the explicit RK3 terms and only the z part implicitly."""
    g = _grid(12, 6, 10, 0.0)
    nu, dt, mx, mz = 0.03, 0.08, 2, 3
    mode, out, _ = _eigen_step(g, "v", mx, mz, nu, dt, implicit)
    lx = -4 / g.dx ** 2 * np.sin(np.pi * mx / g.nx) ** 2
    lz = -4 / g.dzf[0] ** 2 * np.sin(np.pi * mz / (2 * g.nz)) ** 2
    amp, prev = 1.0, 0.0          # amplitude and the carried explicit term of the previous stage
    for a, b, gm in zip(O.RK3_ALPHA, O.RK3_BETA, O.RK3_GAMMA):
        if implicit == 1:
            new = amp * (1 + gm * nu * (lx + lz) * dt / 2) / (1 - gm * nu * (lx + lz) * dt / 2)
        else:
            carry = nu * lx * amp
            new = (amp + dt * (a * carry + b * prev) + gm * nu * lz * dt / 2 * amp) / (1 - gm * nu * lz * dt / 2)
            prev = carry
        amp = new
    assert np.max(np.abs(out - amp * mode)) <= 1e-12


@pytest.mark.parametrize("implicit", [1, 2])
def test_cn_pressure_update_closes_the_momentum_equation(implicit):
    """Eqs. 18-19 (21-22): with p^{k+1/2} - p^{k-1/2} = (I - a L) phi the new
    velocity satisfies (I - a L) u^{k+1} + gamma dt grad(p^{k+1/2} - p^{k-1/2})
    = right-hand side, away from the wall rows where the velocity and the
    pressure take different ghosts."""
    g = _grid(12, 10, 9, 1.7)
    u, v, w = _velocity(101, g)
    p = S.gaussian(104, (g.nz, g.ny, g.nx))
    nut = O.eddy_viscosity(u, v, w, g, 0.1, 1e-3, 0.05)
    nu, dt, stage = 2e-2, 5e-3, 1
    r_prev = O.momentum_rhs(u, v, w, nut, g, nu)
    rhs, _ = O.rk3_rhs(u, v, w, p, nut, r_prev, g, stage, dt, nu, implicit)
    un, vn, wn, pn, _, _ = O.rk3_substep(u, v, w, p, nut, r_prev, g, stage, dt, nu, 0.1, 0.05, implicit)
    gm = O.RK3_GAMMA[stage]
    ah = gm * nu * dt / 2
    parts = O.viscous_parts(un, vn, wn, g)
    gpd = O.gradient(pn - p, g)
    for c, (lxy, lz), gc, rc, rows in zip((un, vn, wn), parts, gpd, rhs,
                                          (slice(1, -1), slice(1, -1), slice(2, -2))):
        lap = lxy + lz if implicit == 1 else lz
        lhs = c - ah * lap + gm * dt * gc
        assert np.max(np.abs((lhs - rc)[rows])) <= 1e-11 * (np.max(np.abs(rc)) + 1.0)


@pytest.mark.parametrize("implicit", [1, 2])
def test_cn_substep_is_divergence_free(implicit):
    g = _grid(12, 8, 10, 1.8)
    u, v, w = _velocity(111, g, divfree=False)
    p = S.gaussian(114, (g.nz, g.ny, g.nx))
    nut = O.eddy_viscosity(u, v, w, g, 0.1, 1e-3, 0.05)
    r = None
    for s in range(3):
        u, v, w, p, nut, r = O.rk3_substep(u, v, w, p, nut, r, g, s, 1e-3, 1e-2, 0.1, 0.05, implicit)
        assert np.max(np.abs(O.divergence(u, v, w, g))) <= 1e-10
        assert np.max(np.abs(w[0])) == 0.0 and np.max(np.abs(w[-1])) == 0.0


def test_mutation_plain_pressure_update_fails_the_coupling_pin(monkeypatch):
    monkeypatch.setattr(R, "laplacian_cell", lambda phi, g, z_only=False: np.zeros_like(phi))
    with pytest.raises(AssertionError):
        test_cn_pressure_update_closes_the_momentum_equation(1)
