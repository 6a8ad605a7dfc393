"""Mode (0, 0) of singular Poisson problems through the z kernel against the
oracle.

With Neumann z sides and only periodic / Neumann x, y sides the (0, 0) line is
singular (Sec. 2.2: the compatibility condition, the pinned last row and the
gauge).  The z kernel solves that line with one warp: the forward elimination
and the back-substitution become affine recurrences (zero pivot excess), run
as shuffle scans over 32 chunks of rows.  These cases cover chunk lengths of
one row and of several rows with a short or empty last chunk (nz = 1, 2, 5,
31, 32, 33, 100, 512), uniform and strongly stretched z, the adjoint solve
(whose line carries the dzf weights), FP64 / FP32 / FP32 + refinement, and the
zero weighted mean of the result (reading R5).  Helmholtz solves of the same
plans take the general path and are checked beside them.

Tolerances as the rest of the suite (relative L2): 1e-12 FP64, 1e-5 FP32,
1e-10 FP32 + refinement.  For nz >= 256 the reference is the oracle's solve
with one FP64 refinement step (reading R13).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu

TOL = {cs.FP64: 1e-12, cs.FP32: 1e-5, cs.FP32_REFINE: 1e-10, cs.FP32_REFINE_FAST: 1e-10}
P, N = O.BC_P, O.BC_N


def pair(nx, ny, nz, bc, beta):
    zf = S.tanh_faces(nz, beta, 2.0)
    odzc, odzf = O.cell_spacings(zf)
    gdzc, gdzf = cs.cell_spacings(zf)
    g = O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, odzc, odzf, bc)
    plan = cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, gdzc, gdzf, cs.FP64, 2)
    return g, plan


def run(plan, f, alpha=None, adjoint=False):
    x = torch.from_numpy(np.ascontiguousarray(f)).to("cuda", plan.dtype)
    if adjoint:
        out = plan.poisson_adjoint(x) if alpha is None else plan.helmholtz_adjoint(alpha, x)
    else:
        out = plan.poisson(x) if alpha is None else plan.helmholtz(alpha, x)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("nz", [1, 2, 5, 31, 32, 33, 100, 512])
@pytest.mark.parametrize("bc", [(P, P, N, N, N, N), (N, N, N, N, N, N)])
@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_singular_line_against_oracle(cuda_device, nz, bc, beta):
    nx, ny = (8, 4) if nz >= 256 else (12, 6)
    g, plan = pair(nx, ny, nz, bc, beta)
    f = S.gaussian(4100 + nz, (nz, ny, nx))          # not projected: the solve removes the mean
    deep = nz >= 256
    ref = O.solve_refined(f, g) if deep else O.solve(f, g)
    for prec in (cs.FP64, cs.FP32, cs.FP32_REFINE, cs.FP32_REFINE_FAST):
        plan.set_precision(prec, 2)
        for rep in range(2):                         # pivots computed, then read from the cache
            p = run(plan, f)
            rel = O.rel_l2(p, ref)
            assert rel <= TOL[prec], (prec, rep, rel)
            assert abs(O.weighted_mean(p, g)) <= 10 * TOL[prec] * np.abs(ref).max(), prec
    plan.set_precision(cs.FP64)
    h = O.solve_refined(f, g, 2e-3) if deep else O.solve(f, g, 2e-3)
    assert O.rel_l2(run(plan, f, 2e-3), h) <= TOL[cs.FP64]
    assert plan.status() == 0


@pytest.mark.parametrize("nz", [2, 33, 100])
@pytest.mark.parametrize("beta", [0.0, 2.0])
def test_singular_line_adjoint_against_oracle(cuda_device, nz, beta):
    bc = (P, P, N, N, N, N)
    g, plan = pair(12, 6, nz, bc, beta)
    w = S.gaussian(4200 + nz, (nz, 6, 12))
    ref = O.solve_T(w, g)
    assert O.rel_l2(run(plan, w, adjoint=True), ref) <= TOL[cs.FP64]
    plan.set_precision(cs.FP32)
    assert O.rel_l2(run(plan, w, adjoint=True), ref) <= TOL[cs.FP32]
    assert plan.status() == 0
