"""Smagorinsky / van Driest eddy viscosity (Eq. 4) through cales_eddy_viscosity
against the oracle, on stretched channel grids."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu


def _pair(nx, ny, nz, precision, beta=1.8):
    zf = S.tanh_faces(nz, beta, 2.0)
    odzc, odzf = O.cell_spacings(zf)
    gdzc, gdzf = cs.cell_spacings(zf)
    bc = (0, 0, 0, 0, 1, 1)
    g = O.Grid(nx, ny, nz, 2 * math.pi / nx, math.pi / ny, odzc, odzf, bc)
    return g, cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, gdzc, gdzf, precision)


def _velocity(seed, nx, ny, nz):
    u = S.gaussian(seed, (nz, ny, nx))
    v = S.gaussian(seed + 1, (nz, ny, nx))
    w = S.gaussian(seed + 2, (nz + 1, ny, nx))
    w[0] = 0.0
    w[-1] = 0.0
    return u, v, w


@pytest.mark.parametrize("shape", [(48, 20, 33), (128, 64, 64), (50, 20, 17), (54, 12, 9)])
@pytest.mark.parametrize("precision,tol", [(cs.FP64, 1e-12), (cs.FP32, 1e-5)])
def test_eddy_viscosity_against_oracle(cuda_device, shape, precision, tol):
    nx, ny, nz = shape
    g, plan = _pair(nx, ny, nz, precision)
    u, v, w = _velocity(8100 + nx, nx, ny, nz)
    dt = plan.dtype
    nut = plan.eddy_viscosity(0.1, 1e-3, 0.06, torch.from_numpy(u).to("cuda", dt),
                              torch.from_numpy(v).to("cuda", dt), torch.from_numpy(w).to("cuda", dt))
    torch.cuda.synchronize()
    ref = O.eddy_viscosity(u, v, w, g, 0.1, 1e-3, 0.06)
    assert O.rel_l2(nut.double().cpu().numpy(), ref) <= tol
    assert np.max(np.abs(nut.double().cpu().numpy() - ref)) <= 10 * tol * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,tol", [(cs.FP64, 1e-12), (cs.FP32, 1e-5)])
def test_eddy_viscosity_unaligned_views(cuda_device, precision, tol):
    """Views one element into their storage: the kernel takes its scalar path."""
    nx, ny, nz = 48, 20, 9
    g, plan = _pair(nx, ny, nz, precision)
    u, v, w = _velocity(8300, nx, ny, nz)
    dt = plan.dtype

    def shifted(x):
        buf = torch.empty(x.size + 1, dtype=dt, device="cuda")
        view = buf[1:].view(x.shape)
        view.copy_(torch.from_numpy(x))
        return view

    out = shifted(np.zeros((nz, ny, nx)))
    nut = plan.eddy_viscosity(0.17, 2e-3, 0.05, shifted(u), shifted(v), shifted(w), out)
    torch.cuda.synchronize()
    assert nut.data_ptr() == out.data_ptr()
    assert O.rel_l2(out.double().cpu().numpy(), O.eddy_viscosity(u, v, w, g, 0.17, 2e-3, 0.05)) <= tol


def test_eddy_viscosity_rejects_bad_arguments(cuda_device):
    _, plan = _pair(16, 8, 8, cs.FP64)
    z = torch.zeros(8, 8, 16, dtype=torch.float64, device="cuda")
    zw = torch.zeros(9, 8, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        plan.eddy_viscosity(0.1, 0.0, 0.05, z, z, zw)            # nu must be positive
    bad = cs.Plan(16, 8, 8, (1, 1, 0, 0, 1, 1), 0.1, 0.1, np.full(9, 0.25), np.full(8, 0.25))
    with pytest.raises(Exception):
        bad.eddy_viscosity(0.1, 1e-3, 0.05, z, z, zw)            # x walls: not a channel plan
