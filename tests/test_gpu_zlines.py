"""Wall-normal implicit step (Eq. 21): (I - alpha L_z) u = f on every line,
through cales_helmholtz_z_solve, against the oracle's per-line Thomas."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu

TOL = {cs.FP64: 1e-12, cs.FP32: 1e-5, cs.FP32_REFINE: 1e-12}


def _pair(nx, ny, nz, bc, precision, beta=1.6):
    face = bc[4] == O.BC_DF or bc[5] == O.BC_DF
    zf = S.tanh_faces(nz + 1 if face else nz, beta, 2.0)
    odzc, odzf = (O.face_spacings if face else O.cell_spacings)(zf)
    gdzc, gdzf = (cs.face_spacings if face else cs.cell_spacings)(zf)
    g = O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, odzc, odzf, bc)
    return g, cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, gdzc, gdzf, precision)


@pytest.mark.parametrize("zlo,zhi", [(1, 1), (2, 2), (2, 1), (1, 2), (3, 3), (2, 3)])
@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32, cs.FP32_REFINE])
def test_z_lines_against_oracle_ragged(cuda_device, zlo, zhi, precision):
    nx, ny, nz = 40, 12, 45            # 480 lines: a partial 32-line tile; 45 rows: uneven segments
    g, plan = _pair(nx, ny, nz, (0, 0, 1, 1, zlo, zhi), precision)
    f = S.gaussian(7100 + 10 * zlo + zhi, (nz, ny, nx))
    x = torch.from_numpy(f).to("cuda", plan.dtype)
    for alpha in (1e-4, 3e-3):
        u = plan.helmholtz_z(alpha, x)
        torch.cuda.synchronize()
        assert O.rel_l2(u.double().cpu().numpy(), O.solve_z_lines(f, g, alpha)) <= TOL[precision], alpha
    assert plan.status() == 0


def test_z_lines_full_segments_in_place_and_identity(cuda_device):
    nx, ny, nz = 64, 32, 512           # the bench's wall-normal depth: full 32-row segments
    g, plan = _pair(nx, ny, nz, (0, 0, 1, 1, 2, 2), cs.FP32_REFINE, beta=1.5)
    f = S.gaussian(7200, (nz, ny, nx))
    x = torch.from_numpy(f).cuda()
    plan.helmholtz_z(2e-4, x, out=x)
    torch.cuda.synchronize()
    assert O.rel_l2(x.cpu().numpy(), O.solve_z_lines(f, g, 2e-4)) <= 1e-12
    y = torch.from_numpy(f).cuda()
    assert torch.equal(plan.helmholtz_z(0.0, y), y)
    plan.set_precision(cs.FP32)
    u32 = plan.helmholtz_z(2e-4, torch.from_numpy(f).cuda().float())
    torch.cuda.synchronize()
    assert O.rel_l2(u32.double().cpu().numpy(), O.solve_z_lines(f, g, 2e-4)) <= 1e-5


def test_z_lines_rejects_negative_alpha(cuda_device):
    _, plan = _pair(16, 8, 8, (0, 0, 1, 1, 1, 1), cs.FP64)
    with pytest.raises(Exception):
        plan.helmholtz_z(-1.0, torch.zeros(8, 8, 16, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32])
def test_z_lines_pivot_cache_follows_alpha(cuda_device, precision):
    """The line solves keep one set of segment-entry pivots (shared by all
    lines) for the last alpha: a sequence of alphas on one plan matches fresh
    plans bit for bit."""
    nx, ny, nz = 48, 16, 300
    bc = (0, 0, 1, 1, 2, 1)
    _, plan = _pair(nx, ny, nz, bc, precision)
    f = torch.from_numpy(S.gaussian(7300, (nz, ny, nx))).to("cuda", plan.dtype)
    for alpha in (1e-3, 1e-3, 5e-4, 1e-3):
        got = plan.helmholtz_z(alpha, f)
        _, fresh = _pair(nx, ny, nz, bc, precision)
        want = fresh.helmholtz_z(alpha, f)
        torch.cuda.synchronize()
        assert torch.equal(got, want), alpha
