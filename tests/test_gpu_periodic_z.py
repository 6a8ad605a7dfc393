"""Periodic z (cyclic tridiagonal per mode) through the C ABI against the
oracle: FP64, FP32 and FP32 + refinement Poisson and Helmholtz solves on
stretched periodic grids, every x/y kind, ragged sizes, the singular
all-periodic case, the FP64 residual, the adjoint and the wall-normal line
solves, and the one path that refuses a periodic z."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu

TOL = {cs.FP64: 1e-12, cs.FP32: 1e-5}


def _periodic(dzc_dzf):
    dzc, dzf = dzc_dzf
    dzc = np.array(dzc, dtype=np.float64)
    dzc[0] = dzc[-1] = 0.5 * (dzf[0] + dzf[-1])            # last centre to first through the period
    return dzc, dzf


def pair(nx, ny, nz, bcx, bcy, beta=1.5, precision=cs.FP64):
    zf = S.tanh_faces(nz, beta, 2.0)
    bc = (bcx, bcx, bcy, bcy, O.BC_P, O.BC_P)
    odzc, odzf = _periodic(O.cell_spacings(zf))
    gdzc, gdzf = _periodic(cs.cell_spacings(zf))
    g = O.Grid(nx, ny, nz, 2 * math.pi / nx, 1.3 / ny, odzc, odzf, bc)
    return g, cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, 1.3 / ny, gdzc, gdzf, precision)


@pytest.mark.parametrize("shape", [(48, 20, 33), (64, 32, 64), (16, 1, 3)])
@pytest.mark.parametrize("bcx,bcy", [(O.BC_P, O.BC_P), (O.BC_P, O.BC_N), (O.BC_N, O.BC_D), (O.BC_D, O.BC_P)])
@pytest.mark.parametrize("alpha", [None, 2e-3])
@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32])
def test_periodic_z_against_oracle(cuda_device, shape, bcx, bcy, alpha, precision):
    nx, ny, nz = shape
    g, plan = pair(nx, ny, nz, bcx, bcy, precision=precision)
    f = S.gaussian(700 + nx + nz + bcx * 3 + bcy, (nz, ny, nx))
    x = torch.from_numpy(f).to("cuda", plan.dtype)
    out = plan.poisson(x) if alpha is None else plan.helmholtz(alpha, x)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    ref = O.solve(f, g, alpha)
    rel = O.rel_l2(got, ref)
    print(f"periodic z {shape} bc {bcx},{bcy} alpha {alpha} prec {precision}: rel {rel:.3e}")
    assert rel <= TOL[precision]
    if O.is_singular(g, alpha):
        assert abs(O.weighted_mean(got, g)) <= (1e-10 if precision == cs.FP64 else 1e-6) * np.max(np.abs(ref))


def test_periodic_z_in_place_and_repeatable(cuda_device):
    g, plan = pair(32, 16, 24, O.BC_P, O.BC_P)
    f = S.gaussian(760, (24, 16, 32))
    x = torch.from_numpy(f).cuda()
    y = plan.poisson(x.clone())
    x2 = x.clone()
    plan.poisson(x2, x2)
    torch.cuda.synchronize()
    assert torch.equal(x2, y)
    assert O.rel_l2(y.cpu().numpy(), O.solve(f, g)) <= TOL[cs.FP64]


@pytest.mark.parametrize("shape", [(48, 20, 33), (64, 32, 64)])
@pytest.mark.parametrize("bcx,bcy", [(O.BC_P, O.BC_P), (O.BC_P, O.BC_N), (O.BC_N, O.BC_D)])
@pytest.mark.parametrize("alpha", [None, 2e-3])
def test_periodic_z_refinement_against_oracle(cuda_device, shape, bcx, bcy, alpha):
    """FP32 solves with double-float refinement over a periodic z: the
    residual wraps through the period, the consistency constant of a
    singular problem is accumulated by the cyclic solve."""
    nx, ny, nz = shape
    g, plan = pair(nx, ny, nz, bcx, bcy, precision=cs.FP32_REFINE)
    f = S.gaussian(720 + nx + nz + bcx * 3 + bcy, (nz, ny, nx))
    x = torch.from_numpy(f).cuda()
    out = plan.poisson(x) if alpha is None else plan.helmholtz(alpha, x)
    torch.cuda.synchronize()
    ref = O.solve(f, g, alpha)
    rel = O.rel_l2(out.cpu().numpy(), ref)
    print(f"periodic z refine {shape} bc {bcx},{bcy} alpha {alpha}: rel {rel:.3e}")
    assert rel <= 1e-10
    assert plan.status() == 0


def test_periodic_z_fp64_residual(cuda_device):
    g, plan = pair(24, 10, 9, O.BC_P, O.BC_N)
    u, f = S.gaussian(740, (9, 10, 24)), S.gaussian(741, (9, 10, 24))
    for alpha in (None, 1e-3):
        r = plan.residual(torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda(), alpha)
        torch.cuda.synchronize()
        ref = O.residual(u, f, g, alpha)
        assert np.abs(r.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32])
@pytest.mark.parametrize("alpha", [1e-3, 0.05])
def test_periodic_z_line_solves(cuda_device, precision, alpha):
    """Wall-normal implicit line solves (Eq. 21) over a periodic z: one cyclic
    system per (i, j) line, out of place and in place."""
    g, plan = pair(24, 10, 33, O.BC_P, O.BC_N, precision=precision)
    f = S.gaussian(750, (33, 10, 24))
    x = torch.from_numpy(f).to("cuda", plan.dtype)
    u = plan.helmholtz_z(alpha, x)
    y = x.clone()
    plan.helmholtz_z(alpha, y, y)
    torch.cuda.synchronize()
    ref = O.solve_z_lines(f, g, alpha)
    assert torch.equal(u, y)
    assert O.rel_l2(u.double().cpu().numpy(), ref) <= TOL[precision]


@pytest.mark.parametrize("bcx,bcy", [(O.BC_P, O.BC_P), (O.BC_N, O.BC_D)])
@pytest.mark.parametrize("alpha", [None, 2e-3])
@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32])
def test_periodic_z_adjoint_matches_oracle_transpose(cuda_device, bcx, bcy, alpha, precision):
    g, plan = pair(48, 20, 33, bcx, bcy, precision=precision)
    w = S.gaussian(760 + bcx, (33, 20, 48))
    x = torch.from_numpy(w).to("cuda", plan.dtype)
    out = plan.poisson_adjoint(x) if alpha is None else plan.helmholtz_adjoint(alpha, x)
    torch.cuda.synchronize()
    rel = O.rel_l2(out.double().cpu().numpy(), O.solve_T(w, g, alpha))
    print(f"periodic z adjoint bc {bcx},{bcy} alpha {alpha} prec {precision}: rel {rel:.3e}")
    assert rel <= TOL[precision]


def test_periodic_z_allocation_free_solve_refuses(cuda_device):
    """The allocation-free entry point keeps to wall-bounded z (its static
    scratch has no room for the cyclic solve's two fields)."""
    import ctypes as C
    from paper_2411_09364_gb300 import _native as N
    g, plan = pair(16, 8, 8, O.BC_P, O.BC_P)
    f = torch.zeros((8, 8, 16), dtype=torch.float64, device="cuda")
    p = torch.zeros_like(f)
    rc = N.lib().cales_poisson_solve_noalloc(plan.handle, C.c_void_p(f.data_ptr()), C.c_void_p(p.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -2
