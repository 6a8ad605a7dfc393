"""GPU parity of the CUDA solver against the FP64 CPU oracle.

Tolerances (relative L2 over all points, both sides gauged): 1e-12 for FP64,
1e-5 for plain FP32, 1e-10 for FP32 + FP64 refinement.
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


def _faces(nz, beta, bc, lz=2.0):
    face = bc[4] == O.BC_DF or bc[5] == O.BC_DF
    zf = S.tanh_faces(nz + 1 if face else nz, beta, lz)
    return zf, face


def pair(nx, ny, nz, bc, beta=1.6, lx=2 * math.pi, ly=math.pi, lz=2.0, precision=cs.FP64, sweeps=2):
    """(oracle grid, GPU plan) on the same synthetic geometry, spacings derived independently."""
    zf, face = _faces(nz, beta, bc, lz)
    odzc, odzf = (O.face_spacings if face else O.cell_spacings)(zf)
    gdzc, gdzf = (cs.face_spacings if face else cs.cell_spacings)(zf)
    g = O.Grid(nx, ny, nz, lx / nx, ly / ny, odzc, odzf, bc)
    plan = cs.Plan(nx, ny, nz, bc, lx / nx, ly / ny, gdzc, gdzf, precision, sweeps)
    return g, plan


def gpu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def solve_gpu(plan, f, alpha=None, adjoint=False):
    x = gpu(f, plan.dtype)
    if adjoint:
        out = plan.poisson_adjoint(x) if alpha is None else plan.helmholtz_adjoint(alpha, x)
    else:
        out = plan.poisson(x) if alpha is None else plan.helmholtz(alpha, x)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def test_config1_channel_fp64(cuda_device):
    nx, ny, nz = 64, 32, 32
    g, plan = pair(nx, ny, nz, (0, 0, 0, 0, 1, 1), beta=0.0)
    f = S.remove_mean(S.uniform(1000, (nz, ny, nx)))
    p = solve_gpu(plan, f)
    ref = O.solve(f, g)
    assert O.rel_l2(p, ref) <= 1e-12
    assert abs(O.weighted_mean(p, g)) <= 1e-14 * np.abs(ref).max()
    assert plan.status() == 0


BCS_XY = (O.BC_P, O.BC_N, O.BC_D)
BCS_Z = [(1, 1), (2, 2), (3, 3), (1, 2), (2, 3), (3, 1)]


@pytest.mark.parametrize("kx,ky", list(itertools.product(BCS_XY, BCS_XY)))
@pytest.mark.parametrize("zlo,zhi", BCS_Z)
@pytest.mark.parametrize("alpha", [None, 3e-3])
def test_bc_matrix_fp64_ragged(cuda_device, kx, ky, zlo, zhi, alpha):
    """All boundary kinds; nx = 40 leaves a ragged column tile, nz = 13 is odd."""
    nx, ny, nz = 40, 12, 13
    bc = (kx, kx, ky, ky, zlo, zhi)
    g, plan = pair(nx, ny, nz, bc)
    f = S.gaussian(11 + kx * 3 + ky, (nz, ny, nx))
    assert O.rel_l2(solve_gpu(plan, f, alpha), O.solve(f, g, alpha)) <= TOL[cs.FP64]


@pytest.mark.parametrize("nx,ny,nz", [(1, 1, 40), (2, 1, 9), (1, 6, 7), (8, 2, 1), (2, 2, 2), (30, 10, 3),
                                      (96, 80, 5), (160, 12, 4)])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0, 1, 1), (1, 1, 2, 2, 2, 3), (2, 2, 1, 1, 1, 2)])
def test_degenerate_and_mixed_radix_sizes(cuda_device, nx, ny, nz, bc):
    g, plan = pair(nx, ny, nz, bc)
    f = S.gaussian(5, (nz, ny, nx))
    for alpha in (None, 1e-2):
        assert O.rel_l2(solve_gpu(plan, f, alpha), O.solve(f, g, alpha)) <= TOL[cs.FP64]


@pytest.mark.parametrize("bc", [(0, 0, 0, 0, 1, 1), (0, 0, 1, 1, 1, 1), (1, 1, 2, 2, 3, 3)])
@pytest.mark.parametrize("alpha", [None, 1e-3])
def test_fp32_and_refinement(cuda_device, bc, alpha):
    nx, ny, nz = 96, 48, 40
    g, plan = pair(nx, ny, nz, bc, beta=1.8)
    f = S.gaussian(21, (nz, ny, nx))
    ref = O.solve(f, g, alpha)
    plan.set_precision(cs.FP32)
    assert O.rel_l2(solve_gpu(plan, f, alpha), ref) <= TOL[cs.FP32]
    plan.set_precision(cs.FP32_REFINE, 2)
    assert O.rel_l2(solve_gpu(plan, f, alpha), ref) <= TOL[cs.FP32_REFINE]


@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32, cs.FP32_REFINE])
def test_pivot_cache_follows_the_operator(cuda_device, precision):
    """The z sweeps keep the segment-entry pivots of the last (sigma, alpha):
    a sequence of solves with changing operators on one plan matches fresh
    plans bit for bit, and the oracle to the precision's tolerance."""
    nx, ny, nz = 64, 32, 300          # 300 rows: several z segments per mode
    bc = (0, 0, 1, 1, 1, 1)
    g, plan = pair(nx, ny, nz, bc, beta=1.8, precision=precision)
    f = S.gaussian(31, (nz, ny, nx))
    for alpha in (1e-3, 2e-4, None, 1e-3, None):
        got = solve_gpu(plan, f, alpha)
        _, fresh = pair(nx, ny, nz, bc, beta=1.8, precision=precision)
        want = solve_gpu(fresh, f, alpha)
        if alpha is None and precision == cs.FP32_REFINE:
            # singular Poisson: the refinement's gauge sum is an atomic FP64 reduction
            assert O.rel_l2(got, want) <= 1e-13, alpha
        else:
            assert np.array_equal(got, want), alpha
        assert O.rel_l2(got, O.solve(f, g, alpha)) <= TOL[precision], alpha


def test_in_place(cuda_device):
    g, plan = pair(48, 24, 20, (0, 0, 1, 1, 1, 1))
    f = S.gaussian(3, (20, 24, 48))
    x = gpu(f)
    plan.poisson(x, out=x)
    torch.cuda.synchronize()
    assert O.rel_l2(x.cpu().numpy(), O.solve(f, g)) <= TOL[cs.FP64]


@pytest.mark.parametrize("bc", [(0, 0, 0, 0, 1, 1), (1, 1, 0, 0, 2, 3), (2, 2, 1, 1, 1, 2)])
@pytest.mark.parametrize("alpha", [None, 2e-3])
def test_adjoint_against_oracle_transpose(cuda_device, bc, alpha):
    nx, ny, nz = 32, 16, 24
    g, plan = pair(nx, ny, nz, bc, beta=1.8)
    w = S.gaussian(31, (nz, ny, nx))
    ref = O.solve_T(w, g, alpha)
    assert O.rel_l2(solve_gpu(plan, w, alpha, adjoint=True), ref) <= TOL[cs.FP64]
    plan.set_precision(cs.FP32)
    assert O.rel_l2(solve_gpu(plan, w, alpha, adjoint=True), ref) <= TOL[cs.FP32]


def test_residual_kernel_matches_oracle(cuda_device):
    for bc, alpha in [((0, 0, 0, 0, 1, 1), None), ((1, 1, 2, 2, 2, 3), 1e-2), ((2, 2, 0, 0, 3, 1), None)]:
        g, plan = pair(24, 20, 16, bc)
        u = S.gaussian(1, (16, 20, 24))
        f = S.gaussian(2, (16, 20, 24))
        r = plan.residual(gpu(u), gpu(f), alpha).cpu().numpy()
        ref = O.residual(u, f, g, alpha)
        assert np.abs(r - ref).max() <= 1e-12 * np.abs(ref).max()


def test_nonfinite_input_sets_status(cuda_device):
    g, plan = pair(16, 8, 8, (0, 0, 0, 0, 2, 2))
    f = np.zeros((8, 8, 16))
    f[3, 2, 1] = np.nan
    solve_gpu(plan, f)
    assert plan.status() & 1
    assert plan.status() == 0      # reading clears the word


def test_config2_channel_divergence_fp64_fp32(cuda_device):
    """512 x 256 x 192, tanh beta = 1.8, RHS = divergence of a Gaussian
    staggered velocity (walls impermeable)."""
    from paper_2411_09364_gb300 import autograd as AG
    nx, ny, nz = 512, 256, 192
    g, plan = pair(nx, ny, nz, (0, 0, 0, 0, 1, 1), beta=1.8)
    u, v, w = S.velocity_field(2000, nx, ny, nz)
    ref = O.solve(O.divergence(u, v, w, g), g)
    f = AG.divergence(plan, gpu(u), gpu(v), gpu(w)).cpu().numpy()    # the GPU's own divergence
    err64 = O.rel_l2(solve_gpu(plan, f), ref)
    plan.set_precision(cs.FP32)
    err32 = O.rel_l2(solve_gpu(plan, f), ref)
    print(f"config2 rel err FP64 {err64:.3e} FP32 {err32:.3e}")
    assert err64 <= TOL[cs.FP64]
    assert err32 <= TOL[cs.FP32]


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("zvariant", [0, 1])
@pytest.mark.parametrize("bc,nx,ny", [((0, 0, 1, 1, 1, 2), 480, 120), ((1, 2, 3, 3, 1, 1), 480, 119)])
def test_schedule_radix_order_and_z_variant(cuda_device, order, zvariant, bc, nx, ny):
    """Every FFT radix order (radix 16 first, 5 and 3 first, radix 8 only) and
    both z kernel variants of the launch schedule solve the same system:
    lengths with factors 2, 3 and 5 (x 480 = 2 x 240; y 120 = 2 x 60, or 119
    node unknowns: FFT length 120), Neumann, mixed and node kinds, in FP64,
    FP32 and FP32 + refinement."""
    nz = 48
    g, plan = pair(nx, ny, nz, bc, beta=1.7)
    plan.set_schedule([0, 0, 0, 0, order, zvariant])
    assert plan.schedule()[4:] == (order, zvariant)
    f = S.gaussian(71 + order, (nz, ny, nx))
    for alpha in (None, 1e-3):
        ref = O.solve(f, g, alpha)
        for prec in (cs.FP64, cs.FP32, cs.FP32_REFINE):
            plan.set_precision(prec, 2)
            assert O.rel_l2(solve_gpu(plan, f, alpha), ref) <= TOL[prec], (prec, alpha)
    assert plan.status() == 0


@pytest.mark.parametrize("bc", [(0, 0, 0, 0, 1, 1), (0, 0, 1, 1, 1, 1), (1, 1, 2, 2, 3, 3), (1, 2, 0, 0, 2, 1),
                                (3, 3, 2, 1, 1, 3), (0, 0, 0, 0, 0, 0)])
@pytest.mark.parametrize("alpha", [None, 1e-3])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_fast_refinement_against_oracle(cuda_device, bc, alpha, sweeps):
    """FP32 solves with one double-float residual and FP32 residual updates
    for the later sweeps: every z kind (periodic included, with its wrap
    distance), mixed and node-centred x/y kinds, Poisson and Helmholtz, two
    and three sweeps, within the refinement tolerance of the oracle."""
    nx = 95 if bc[0] == 3 else 96
    ny, nz = 48, 40
    if bc[4] == 0:
        zf = S.tanh_faces(nz, 1.6, 2.0)
        odzc, odzf = O.cell_spacings(zf)
        gdzc, gdzf = cs.cell_spacings(zf)
        odzc = np.array(odzc)
        gdzc = np.array(gdzc)
        odzc[0] = odzc[-1] = gdzc[0] = gdzc[-1] = 0.5 * (gdzf[0] + gdzf[-1])
        g = O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, odzc, odzf, bc)
        plan = cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, gdzc, gdzf)
    else:
        g, plan = pair(nx, ny, nz, bc, beta=1.8)
    plan.set_precision(cs.FP32_REFINE_FAST, sweeps)
    f = S.gaussian(81 + sweeps, (nz, ny, nx))
    rel = O.rel_l2(solve_gpu(plan, f, alpha), O.solve(f, g, alpha))
    print(f"fast refinement bc {bc} alpha {alpha} sweeps {sweeps}: rel {rel:.3e}")
    # one sweep is the plain refinement (nothing to update): about 1e-10
    assert rel <= (TOL[cs.FP32_REFINE] if sweeps > 1 else 1e-9), rel
    assert plan.status() == 0
