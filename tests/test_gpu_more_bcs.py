"""The remaining boundary kinds of the uniform directions through the C ABI
against the oracle: node-centred unknowns between two wall nodes (DST-I) and
mixed Neumann / Dirichlet sides (DCT-IV, DST-IV), alone and combined with the
other kinds, in FP64, FP32 and FP32 + refinement; Poisson, Helmholtz, the
adjoint solve and the FP64 residual; degenerate one- and two-point lines; and
the transform lengths that have compile-time kernels for the other kinds.

Tolerances as the rest of the suite (relative L2 over all points): 1e-12
FP64, 1e-5 FP32, 1e-10 FP32 + refinement.
"""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu

TOL = {cs.FP64: 1e-12, cs.FP32: 1e-5, cs.FP32_REFINE: 1e-10}
P, N, D, DF = O.BC_P, O.BC_N, O.BC_D, O.BC_DF
SIDES = [(P, P), (N, N), (D, D), (DF, DF), (N, D), (D, N)]
NEW = [(DF, DF), (N, D), (D, N)]


def _len(sides, even, node):
    """A line length the transform takes: n + 1 factorable for node unknowns,
    an even n with a factorable half otherwise."""
    return node if sides == (DF, DF) else even


def pair(nx, ny, nz, bc, beta=1.6, lx=2 * math.pi, ly=math.pi, precision=cs.FP64, sweeps=2):
    face = bc[4] == DF or bc[5] == DF
    zf = S.tanh_faces(nz + 1 if face else nz, beta, 2.0)
    odzc, odzf = (O.face_spacings if face else O.cell_spacings)(zf)
    gdzc, gdzf = (cs.face_spacings if face else cs.cell_spacings)(zf)
    g = O.Grid(nx, ny, nz, lx / nx, ly / ny, odzc, odzf, bc)
    plan = cs.Plan(nx, ny, nz, bc, lx / nx, ly / ny, gdzc, gdzf, precision, sweeps)
    return g, plan


def solve_gpu(plan, f, alpha=None, adjoint=False):
    x = torch.from_numpy(np.ascontiguousarray(f)).to("cuda", plan.dtype)
    if adjoint:
        out = plan.poisson_adjoint(x) if alpha is None else plan.helmholtz_adjoint(alpha, x)
    else:
        out = plan.poisson(x) if alpha is None else plan.helmholtz(alpha, x)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


COMBOS = [(sx, sy) for sx, sy in itertools.product(SIDES, SIDES) if sx in NEW or sy in NEW]


@pytest.mark.parametrize("sx,sy", COMBOS)
@pytest.mark.parametrize("zlo,zhi", [(N, N), (D, DF)])
@pytest.mark.parametrize("alpha", [None, 3e-3])
def test_new_kinds_fp64(cuda_device, sx, sy, zlo, zhi, alpha):
    """Every pairing of a new kind with every other kind; ragged sizes (40 or
    39 columns leave a partial y tile, 13 z cells)."""
    nx, ny, nz = _len(sx, 40, 39), _len(sy, 12, 11), 13
    bc = (*sx, *sy, zlo, zhi)
    g, plan = pair(nx, ny, nz, bc)
    f = S.gaussian(600 + 7 * SIDES.index(sx) + SIDES.index(sy), (nz, ny, nx))
    rel = O.rel_l2(solve_gpu(plan, f, alpha), O.solve(f, g, alpha))
    assert rel <= TOL[cs.FP64], rel
    assert plan.status() == 0


@pytest.mark.parametrize("sx,sy,nx,ny", [
    ((N, D), (D, N), 96, 48), ((DF, DF), (N, D), 95, 48), ((D, N), (DF, DF), 96, 47),
    ((N, D), (N, N), 1536, 16),      # x length of the compile-time periodic rows, mixed kind
    ((P, P), (N, D), 64, 512),       # y length of the one-buffer column kernel, mixed kind
    ((P, P), (DF, DF), 64, 511),     # node unknowns, FFT length 512
])
@pytest.mark.parametrize("alpha", [None, 1e-3])
def test_new_kinds_fp32_and_refinement(cuda_device, sx, sy, nx, ny, alpha):
    nz = 24
    bc = (*sx, *sy, N, N)
    g, plan = pair(nx, ny, nz, bc, beta=1.8)
    f = S.gaussian(650 + nx + ny, (nz, ny, nx))
    ref = O.solve(f, g, alpha)
    for prec in (cs.FP32, cs.FP32_REFINE, cs.FP64):
        plan.set_precision(prec, 2)
        rel = O.rel_l2(solve_gpu(plan, f, alpha), ref)
        assert rel <= TOL[prec], (prec, rel)
    assert plan.status() == 0


@pytest.mark.parametrize("nx,ny,nz,bc", [
    (1, 6, 5, (N, D, N, D, N, N)), (1, 1, 7, (DF, DF, D, N, N, N)), (2, 4, 3, (DF, DF, DF, DF, D, D)),
    (2, 2, 2, (D, N, N, D, N, N)), (5, 4, 4, (DF, DF, N, D, D, D)), (6, 1, 9, (N, D, N, N, N, D)),
])
def test_new_kinds_degenerate_lengths(cuda_device, nx, ny, nz, bc):
    g, plan = pair(nx, ny, nz, bc)
    f = S.gaussian(670 + nx * ny, (nz, ny, nx))
    for alpha in (None, 1e-2):
        assert O.rel_l2(solve_gpu(plan, f, alpha), O.solve(f, g, alpha)) <= TOL[cs.FP64]


@pytest.mark.parametrize("bc", [(N, D, DF, DF, N, N), (DF, DF, D, N, D, D), (D, N, N, D, N, DF)])
@pytest.mark.parametrize("alpha", [None, 2e-3])
def test_new_kinds_adjoint_matches_oracle_transpose(cuda_device, bc, alpha):
    nx = 39 if bc[0] == DF else 40
    ny = 11 if bc[2] == DF else 12
    nz = 10
    g, plan = pair(nx, ny, nz, bc)
    w = S.gaussian(690, (nz, ny, nx))
    assert O.rel_l2(solve_gpu(plan, w, alpha, adjoint=True), O.solve_T(w, g, alpha)) <= TOL[cs.FP64]
    plan.set_precision(cs.FP32)
    assert O.rel_l2(solve_gpu(plan, w, alpha, adjoint=True), O.solve_T(w, g, alpha)) <= TOL[cs.FP32]


@pytest.mark.parametrize("bc", [(N, D, DF, DF, N, D), (DF, DF, N, D, DF, N), (D, N, D, N, D, D)])
def test_new_kinds_fp64_residual(cuda_device, bc):
    nx = 39 if bc[0] == DF else 40
    ny = 11 if bc[2] == DF else 12
    nz = 9
    g, plan = pair(nx, ny, nz, bc)
    u = S.gaussian(700, (nz, ny, nx))
    f = S.gaussian(701, (nz, ny, nx))
    for alpha in (None, 1e-3):
        ud, fd = (torch.from_numpy(a).cuda() for a in (u, f))
        r = plan.residual(ud, fd, alpha)
        torch.cuda.synchronize()
        ref = O.residual(u, f, g, alpha)
        assert np.abs(r.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
