"""The last residual update of the fast refinement fused into the forward x
transform, against the standalone update kernel followed by the plain
transform.

Both form the update with the same device function and run the same transform
steps on the same rows, so the solves agree bit for bit.  The fused path (off
by default: slower on GB300) runs in a child process started with
CALES_FUSE_RU=1 (read once per process).
Cases: the bench's duct family (periodic x of 1536, Neumann y and z), a
singular channel, Dirichlet and wall-node z with Helmholtz, periodic z, two
and three sweeps, and a row length that is not a multiple of four (no fusion
there: both processes run the standalone update).
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synth_inputs as S
from paper_2411_09364_gb300 import solver as cs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (nx, ny, nz, bc, beta, sweeps)
CASES = [
    (1536, 64, 24, (0, 0, 1, 1, 1, 1), 1.5, 2),      # the bench's duct family
    (128, 64, 40, (0, 0, 0, 0, 1, 1), 1.8, 3),       # singular channel, three sweeps
    (96, 48, 40, (1, 1, 2, 2, 3, 3), 1.7, 2),        # Neumann x, Dirichlet y, wall-node z
    (96, 48, 32, (0, 0, 0, 0, 0, 0), 1.6, 2),        # periodic z
    (90, 48, 32, (0, 0, 1, 1, 2, 2), 1.6, 2),        # rows of 90 points: standalone update in both
]


def _solve_all():
    out = {}
    for ci, (nx, ny, nz, bc, beta, sweeps) in enumerate(CASES):
        zf = S.tanh_faces(nz, beta, 2.0)
        dzc, dzf = cs.cell_spacings(zf)
        if bc[4] == 0:
            dzc = np.array(dzc)
            dzc[0] = dzc[-1] = 0.5 * (dzf[0] + dzf[-1])
        plan = cs.Plan(nx, ny, nz, bc, 2 * math.pi / nx, math.pi / ny, dzc, dzf, cs.FP32_REFINE_FAST, sweeps)
        f = torch.from_numpy(S.gaussian(9700 + ci, (nz, ny, nx))).cuda()
        for alpha in (None, 1e-3):
            u = plan.poisson(f) if alpha is None else plan.helmholtz(alpha, f)
            torch.cuda.synchronize()
            out[f"{ci}_{alpha}"] = u.cpu().numpy()
        assert plan.status() == 0
    return out


def test_fused_and_standalone_residual_update_agree_bitwise(cuda_device, tmp_path):
    mine = _solve_all()
    dst = tmp_path / "fused.npz"
    code = ("import sys, numpy as np; sys.path.insert(0, %r); "
            "import tests.test_gpu_fused_update as T; np.savez(%r, **T._solve_all())" % (ROOT, str(dst)))
    env = dict(os.environ, CALES_FUSE_RU="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    other = np.load(dst)
    for k, v in mine.items():
        w = other[k]
        ci, alpha = k.split("_")
        bc = CASES[int(ci)][3]
        if all(b in (0, 1) for b in bc) and alpha == "None":
            # singular Poisson: the gauge sum of the refinement is an FP64 atomic reduction
            assert np.linalg.norm(v - w) <= 1e-13 * np.linalg.norm(w), k
        else:
            assert np.array_equal(v, w), (k, float(np.abs(v - w).max()))
