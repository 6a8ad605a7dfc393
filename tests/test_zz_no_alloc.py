"""cales_poisson_solve_noalloc: the Poisson solve for callers that cannot
allocate device memory at solve time (a host that gives the library a fixed
memory budget, a time-stepping loop that must not block in the allocator).
It takes its scratch from a static device array of the library instead of
the plan's workspace; its result must match the regular FP32 + refinement
entry point within the refinement tolerance, call after call (the shared
array keeps the previous call's contents).  It runs on plans of any
precision; on an FP32 or FP32 + refinement plan it shares the plan's cache of
FP32 z pivots with the regular solves.

Collected last on purpose (file name), so a failure here stops a ``-x`` run
only after every other test has run.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import synth_inputs as S
from paper_2411_09364_gb300 import _native as N
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu
TOL_REFINE = 1e-10


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _noalloc(plan, f, p):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return N.lib().cales_poisson_solve_noalloc(plan.handle, C.c_void_p(f.data_ptr()), C.c_void_p(p.data_ptr()),
                                               stream)


@pytest.mark.parametrize("bc,beta", [((0, 0, 0, 0, 1, 1), 1.8), ((0, 0, 1, 1, 1, 1), 1.5), ((1, 1, 2, 2, 2, 3), 1.2)])
@pytest.mark.parametrize("noalloc_precision", [cs.FP64, cs.FP32_REFINE])
def test_noalloc_matches_refine_entry_point_twice(cuda_device, bc, beta, noalloc_precision):
    nx, ny, nz = 96, 48, 40
    zf = S.tanh_faces(nz + 1 if bc[5] == 3 else nz, beta)
    dzc, dzf = (cs.face_spacings if bc[5] == 3 else cs.cell_spacings)(zf)
    plan = cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, dzc, dzf, cs.FP32_REFINE, 2)
    noalloc_plan = cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, dzc, dzf, noalloc_precision, 2)
    for seed in (41, 42):
        f = torch.from_numpy(S.gaussian(seed, (nz, ny, nx))).to(cuda_device)
        ref = plan.poisson(f)
        p = torch.full_like(f, float("nan"))
        assert _noalloc(noalloc_plan, f, p) == 0
        torch.cuda.synchronize()
        assert _rel(p, ref) <= TOL_REFINE
    assert noalloc_plan.status() == 0


def test_noalloc_rejects_grids_beyond_its_scratch(cuda_device):
    nx, ny, nz = 1024, 1024, 9          # 9,437,184 points > 8 * 2^20
    dzc, dzf = cs.cell_spacings(S.tanh_faces(nz, 1.0))
    plan = cs.Plan(nx, ny, nz, (0, 0, 0, 0, 1, 1), 1.0 / nx, 1.0 / ny, dzc, dzf)
    f = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    p = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    assert _noalloc(plan, f, p) == -5
    assert b"static scratch" in N.lib().cales_strerror(-5)
