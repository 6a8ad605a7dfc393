"""Parity of the benchmark workload's own kernels with the FP64 CPU oracle.

The benchmark solves the duct Poisson problem of Sec. 2.2 (periodic x with
Lx = 6, Neumann y walls with Ly = 2 -> DCT-II, Neumann z walls stretched by
tanh(beta = 1.5)) at 1536 x 512 x 512 in FP32 with double-float refinement.
Its x rows (n = 1536, L = 768) and y columns (n = 512, L = 256) take the
compile-time-size transform kernels, its z lines (nz = 512) the
warp-per-segment kernel with 16 segments of 32 rows.  These tests drive the
same plan constructor on:

* 1536 x 512 x nz with a thin z (every x/y kernel of the benchmark, the
  oracle's explicit O(n^2) transforms finish in seconds),
* 64 x 32 x 512 (the benchmark's full z depth and its z kernel),
* the full 1536 x 512 x 512 grid with a manufactured solution: p* seeded
  Gaussian with zero dzf-weighted mean (reading R5), f = L p* by the oracle's
  stencil (reading R1/R2).  The method is a direct solver of the discrete
  system, so the exact answer is p* itself; the comparison is element-wise
  over all 402,653,184 points.

Tolerances (relative L2 over all points): 1e-12 FP64, 1e-5 FP32, 1e-10
FP32 + refinement (both refinement modes); the largest point error is bounded by 10x the same
fraction of the largest |p|.  The full-size manufactured case has an FP64
floor of its own: f = L p* is rounded in FP64 with |L p*| up to
4 |p*| (1/dx^2 + 1/dy^2 + 1/dz_min^2) ~ 3e6 |p*|, and the solve returns
L^-1 of that rounding; the oracle's own solve of the same construction at
256 x 128 x 512 and 64 x 32 x 512 stays at 7e-14 .. 1.3e-13, well inside
1e-12.
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
NAMES = {cs.FP64: "FP64", cs.FP32: "FP32", cs.FP32_REFINE: "FP32+refine", cs.FP32_REFINE_FAST: "FP32+fast refine"}
BC = (0, 0, 1, 1, 1, 1)          # P x, N y (DCT-II), N z
LX, LY, LZ, BETA = 6.0, 2.0, 2.0, 1.5


def duct_pair(nx, ny, nz, precision=cs.FP64):
    """(oracle grid, GPU plan) of the benchmark's duct family; the spacings are
    derived independently by each side from the same tanh faces."""
    zf = S.tanh_faces(nz, BETA, LZ)
    odzc, odzf = O.cell_spacings(zf)
    gdzc, gdzf = cs.cell_spacings(zf)
    g = O.Grid(nx, ny, nz, LX / nx, LY / ny, odzc, odzf, BC)
    plan = cs.Plan(nx, ny, nz, BC, LX / nx, LY / ny, gdzc, gdzf, precision, 2)
    return g, plan, zf


def gpu_solve(plan, f_host):
    dt = torch.float32 if plan.precision == cs.FP32 else torch.float64
    f = torch.from_numpy(np.ascontiguousarray(f_host)).to("cuda", dt)
    p = plan.poisson(f)
    torch.cuda.synchronize()
    return p.double().cpu().numpy()


def check(got, ref, precision, what):
    rel = O.rel_l2(got, ref)
    mx = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"{what} {NAMES[precision]}: rel L2 {rel:.3e}, max-abs/max|p| {mx:.3e}")
    assert rel <= TOL[precision], (what, NAMES[precision], rel)
    assert mx <= 10 * TOL[precision], (what, NAMES[precision], mx)


@pytest.mark.parametrize("nz", [16, 9])
def test_bench_xy_kernels_vs_oracle(cuda_device, nz):
    """1536 x 512 x nz duct, seeded Gaussian RHS with its weighted mean
    removed: every x and y kernel of the benchmark (nz = 9 also gives a
    ragged z segment), in all three precisions."""
    nx, ny = 1536, 512
    g, plan, zf = duct_pair(nx, ny, nz)
    f = S.remove_mean(S.gaussian(3000, (nz, ny, nx)), np.diff(zf))
    ref = O.solve(f, g)
    for prec in (cs.FP64, cs.FP32, cs.FP32_REFINE, cs.FP32_REFINE_FAST):
        plan.set_precision(prec, 2)
        check(gpu_solve(plan, f), ref, prec, f"duct {nx}x{ny}x{nz}")
    assert plan.status() == 0


def test_bench_z_depth_vs_oracle(cuda_device):
    """64 x 32 x 512 duct: the benchmark's 512-row stretched z lines (16
    segments of 32 rows, cached segment-entry pivots on the second solve).
    The reference is the oracle's solve with one FP64 refinement step: the
    plain expansion's scalar Thomas sweeps are themselves off by about 1e-12
    on the near-singular modes of this grid (condition numbers near 3e6),
    which is the FP64 tolerance."""
    nx, ny, nz = 64, 32, 512
    g, plan, zf = duct_pair(nx, ny, nz)
    f = S.remove_mean(S.gaussian(3001, (nz, ny, nx)), np.diff(zf))
    ref = O.solve_refined(f, g)
    for prec in (cs.FP64, cs.FP32, cs.FP32_REFINE, cs.FP32_REFINE_FAST):
        plan.set_precision(prec, 2)
        for rep in range(2):                 # first solve fills the pivot cache, second reads it
            check(gpu_solve(plan, f), ref, prec, f"duct {nx}x{ny}x{nz} (solve {rep})")
    assert plan.status() == 0


def test_bench_workload_full_size_manufactured(cuda_device):
    """The benchmark grid itself, 1536 x 512 x 512, through the benchmark's
    plan: f = L p* (oracle stencil) and the solve must return p* at every
    point, in FP32 + refinement (the timed mode), FP64 and FP32."""
    nx, ny, nz = 1536, 512, 512
    zf = S.tanh_faces(nz, BETA, LZ)
    odzc, odzf = O.cell_spacings(zf)
    g = O.Grid(nx, ny, nz, LX / nx, LY / ny, odzc, odzf, BC)
    ps = S.gaussian(3100, (nz, ny, nx))
    ps -= O.weighted_mean(ps, g)
    f = O.apply_L(ps, g)
    gdzc, gdzf = cs.cell_spacings(zf)
    plan = cs.Plan(nx, ny, nz, BC, LX / nx, LY / ny, gdzc, gdzf, cs.FP32_REFINE, 2)
    f_dev = torch.from_numpy(f).cuda()
    del f
    p_dev = torch.empty_like(f_dev)
    for prec in (cs.FP32_REFINE, cs.FP32_REFINE_FAST, cs.FP64, cs.FP32):
        plan.set_precision(prec, 2)
        if prec == cs.FP32:
            f32 = f_dev.float()
            p32 = plan.poisson(f32)
            torch.cuda.synchronize()
            got = p32.double().cpu().numpy()
            del f32, p32
        else:
            plan.poisson(f_dev, p_dev)
            plan.poisson(f_dev, p_dev)       # second solve: cached z pivots, as in the timed loop
            torch.cuda.synchronize()
            got = p_dev.cpu().numpy()
        check(got, ps, prec, f"duct {nx}x{ny}x{nz} manufactured")
        del got
    assert plan.status() == 0
