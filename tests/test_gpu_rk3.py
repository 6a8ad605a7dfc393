"""Explicit RK3 pressure-correction substeps (Eqs. 11-14, then Eq. 4) through
cales_rk3_substep against the oracle: three chained stages on stretched
channels, every output (u, v, w, p, nu_t, R) compared after each stage."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu

NU, CS, UTAU, DT = 2e-3, 0.12, 0.08, 4e-4


def _pair(nx, ny, nz, precision, beta=1.8):
    zf = S.tanh_faces(nz, beta, 2.0)
    odzc, odzf = O.cell_spacings(zf)
    gdzc, gdzf = cs.cell_spacings(zf)
    bc = (0, 0, 0, 0, 1, 1)
    g = O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, odzc, odzf, bc)
    return g, cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, gdzc, gdzf, precision)


def _state(seed, g):
    u = S.gaussian(seed, (g.nz, g.ny, g.nx))
    v = S.gaussian(seed + 1, (g.nz, g.ny, g.nx))
    w = S.gaussian(seed + 2, (g.nz + 1, g.ny, g.nx))
    w[0] = 0.0
    w[-1] = 0.0
    u, v, w = O.project_velocity([u, v, w], g)
    p = S.gaussian(seed + 3, (g.nz, g.ny, g.nx))
    nut = O.eddy_viscosity(u, v, w, g, CS, NU, UTAU)
    return [u, v, w, p, nut]


# (rel-L2 tolerance for u, v, w, nu_t, R; for p)
TOL = {cs.FP64: (1e-11, 1e-10), cs.FP32_REFINE: (1e-11, 1e-10), cs.FP32_REFINE_FAST: (1e-10, 1e-9),
       cs.FP32: (1e-4, 1e-3)}


@pytest.mark.parametrize("shape", [(32, 16, 24), (24, 20, 9)])
@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32_REFINE, cs.FP32_REFINE_FAST, cs.FP32])
def test_rk3_substeps_against_oracle(cuda_device, shape, precision):
    g, plan = _pair(*shape, precision)
    st = _state(9100 + shape[0], g)
    dt = plan.dtype
    dev = [torch.from_numpy(a).to("cuda", dt) for a in st]
    # R^{-1} is not read at stage 0: NaN there must not reach any output
    rdev = [torch.full_like(dev[0], float("nan")), torch.full_like(dev[0], float("nan")),
            torch.full_like(dev[2], float("nan"))]
    work = plan.rk3_work()
    r = None
    tol, tolp = TOL[precision]
    for stage in range(3):
        plan.rk3_substep(stage, DT, NU, CS, UTAU, *dev, *rdev, work)
        torch.cuda.synchronize()
        *st, r = O.rk3_substep(*st, r, g, stage, DT, NU, CS, UTAU)
        got = [t.double().cpu().numpy() for t in dev + rdev]
        want = st + list(r)
        names = ["u", "v", "w", "p", "nut", "ru", "rv", "rw"]
        for name, a, b in zip(names, got, want):
            assert np.all(np.isfinite(a)), (stage, name)
            err = O.rel_l2(a, b)
            assert err <= (tolp if name == "p" else tol), (stage, name, err)
        assert np.max(np.abs(got[2][0])) == 0.0 and np.max(np.abs(got[2][-1])) == 0.0
    # the result is divergence-free to the solver's precision
    d = O.divergence(*got[:3], g)
    assert np.max(np.abs(d)) <= (1e-9 if precision != cs.FP32 else 1e-3)


def test_rk3_substep_rejects_bad_arguments(cuda_device):
    g, plan = _pair(16, 8, 8, cs.FP64)
    n = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    nw = torch.zeros((9, 8, 16), dtype=torch.float64, device="cuda")
    args = [n, n.clone(), nw, n.clone(), n.clone(), n.clone(), n.clone(), nw.clone()]
    with pytest.raises(Exception):
        plan.rk3_substep(3, DT, NU, CS, UTAU, *args)               # stage out of range
    with pytest.raises(Exception):
        plan.rk3_substep(0, 0.0, NU, CS, UTAU, *args)              # dt must be positive
    duct = cs.Plan(16, 8, 8, (0, 0, 1, 1, 1, 1), 0.1, 0.1, np.full(9, 0.25), np.full(8, 0.25))
    with pytest.raises(Exception):
        duct.rk3_substep(0, DT, NU, CS, UTAU, *args)               # not a channel plan


NU_CN, DT_CN = 0.05, 2e-3          # a = gamma nu dt / 2 large enough to matter next to u


@pytest.mark.parametrize("shape", [(32, 16, 24), (24, 20, 9)])
@pytest.mark.parametrize("implicit", [1, 2])
@pytest.mark.parametrize("precision", [cs.FP64, cs.FP32_REFINE, cs.FP32])
def test_rk3_cn_substeps_against_oracle(cuda_device, shape, implicit, precision):
    """Crank-Nicolson substeps: Eqs. 17-19 (implicit = 1, Helmholtz solves)
    and Eqs. 20-22 (implicit = 2, line solves)."""
    nx, ny, nz = shape
    g, plan = _pair(nx, ny, nz, precision)
    uvp, wp = cs.channel_velocity_plans(nx, ny, S.tanh_faces(nz, 1.8, 2.0), 2 * math.pi / nx, math.pi / ny,
                                        precision)
    st = _state(9300 + nx + implicit, g)
    dt = plan.dtype
    dev = [torch.from_numpy(a).to("cuda", dt) for a in st]
    rdev = [torch.full_like(dev[0], float("nan")), torch.full_like(dev[0], float("nan")),
            torch.full_like(dev[2], float("nan"))]
    work = plan.rk3_work()
    r = None
    tol, tolp = TOL[precision]
    for stage in range(3):
        plan.rk3_substep_cn(uvp, wp, implicit, stage, DT_CN, NU_CN, CS, UTAU, *dev, *rdev, work)
        torch.cuda.synchronize()
        *st, r = O.rk3_substep(*st, r, g, stage, DT_CN, NU_CN, CS, UTAU, implicit)
        got = [t.double().cpu().numpy() for t in dev + rdev]
        for name, a, b in zip(["u", "v", "w", "p", "nut", "ru", "rv", "rw"], got, st + list(r)):
            assert np.all(np.isfinite(a)), (stage, name)
            err = O.rel_l2(a, b)
            assert err <= (tolp if name == "p" else tol), (stage, name, err)
        assert np.max(np.abs(got[2][0])) == 0.0 and np.max(np.abs(got[2][-1])) == 0.0
    assert np.max(np.abs(O.divergence(*got[:3], g))) <= (1e-9 if precision != cs.FP32 else 1e-3)


def test_rk3_cn_rejects_mismatched_plans(cuda_device):
    nx, ny, nz = 16, 8, 8
    g, plan = _pair(nx, ny, nz, cs.FP64)
    zf = S.tanh_faces(nz, 1.8, 2.0)
    uvp, wp = cs.channel_velocity_plans(nx, ny, zf, 2 * math.pi / nx, math.pi / ny, cs.FP64)
    n = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    nw = torch.zeros((nz + 1, ny, nx), dtype=torch.float64, device="cuda")
    args = [n, n.clone(), nw, n.clone(), n.clone(), n.clone(), n.clone(), nw.clone()]
    with pytest.raises(Exception):
        plan.rk3_substep_cn(wp, uvp, 1, 0, DT, NU, CS, UTAU, *args)          # plans swapped
    with pytest.raises(Exception):
        plan.rk3_substep_cn(uvp, wp, 3, 0, DT, NU, CS, UTAU, *args)          # no such mode
    uv32, w32 = cs.channel_velocity_plans(nx, ny, zf, 2 * math.pi / nx, math.pi / ny, cs.FP32)
    with pytest.raises(Exception):
        plan.rk3_substep_cn(uv32, w32, 1, 0, DT, NU, CS, UTAU, *args)        # precision differs
