"""Pins of the learned-closure oracle (no GPU)."""
import math

import numpy as np

import oracle as O
import synth_inputs as S

RNG = np.random.default_rng(7)


def _grid(nx=8, ny=6, nz=10, beta=1.8):
    dzc, dzf = O.cell_spacings(S.tanh_faces(nz, beta))
    return O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, dzc, dzf, (0, 0, 0, 0, 1, 1))


def test_stencil_matches_direct_loop():
    g = _grid()
    vel = list(S.velocity_field(11, g.nx, g.ny, g.nz))
    theta = RNG.standard_normal((3, 27))
    out = O.stencil_apply(theta, vel)
    for c, (k, j, i) in [(0, (0, 0, 0)), (1, (9, 5, 7)), (2, (5, 2, 3)), (2, (10, 1, 1)), (0, (4, 5, 0))]:
        a = vel[c]
        nzc = a.shape[0]
        ref = 0.0
        for t in range(27):
            dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
            kk = k + dz
            if 0 <= kk < nzc:
                ref += theta[c, t] * a[kk, (j + dy) % g.ny, (i + dx) % g.nx]
        if c == 2 and k in (0, nzc - 1):
            ref = 0.0
        assert math.isclose(out[c][k, j, i], ref, rel_tol=1e-12, abs_tol=1e-12)


def test_loss_gradient_matches_central_differences():
    g = _grid()
    vel = list(S.velocity_field(5, g.nx, g.ny, g.nz))
    target = O.project_velocity(O.hidden_operator(vel), g)
    theta = 0.05 * RNG.standard_normal((3, 27))
    loss, grad = O.closure_loss_grad(theta, vel, target, g)
    assert math.isclose(loss, O.closure_loss(theta, vel, target, g), rel_tol=1e-12)
    eps = 1e-4
    for c, t in [(0, 13), (1, 0), (2, 26), (2, 13), (1, 17), (0, 4)]:
        tp = theta.copy()
        tp[c, t] += eps
        tm = theta.copy()
        tm[c, t] -= eps
        fd = (O.closure_loss(tp, vel, target, g) - O.closure_loss(tm, vel, target, g)) / (2 * eps)
        assert math.isclose(grad[c, t], fd, rel_tol=1e-6, abs_tol=1e-10)


def test_hidden_operator_is_learnable_by_exact_stencil():
    """With beta = 0 the hidden map is a 27-tap stencil: the loss at the true
    parameters is zero, so a stencil closure can represent it."""
    g = _grid()
    vel = list(S.velocity_field(9, g.nx, g.ny, g.nz))
    target = O.project_velocity(O.hidden_operator(vel, beta=0.0), g)
    theta = np.full((3, 27), O.HIDDEN_KAPPA / 26.0)
    theta[:, 13] = -O.HIDDEN_KAPPA
    assert O.closure_loss(theta, vel, target, g) < 1e-25
    assert O.closure_loss(np.zeros((3, 27)), vel, target, g) > 1e-3
