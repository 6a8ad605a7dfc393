"""The persistent double-buffered z kernel against the one-tile-per-CTA kernel.

Both run the same per-tile arithmetic (the same device function), so their
solves agree bit for bit.  The persistent kernel runs in a child process started
with CALES_ZPERSIST=1 (read once per process).  The grids have enough modes
(at least eight 32-mode tiles per SM) for the persistent kernel to be chosen:
full and ragged z segments, a ragged last mode tile, the bench's 512-deep duct
lines (16 segments of 32 rows, singular mode (0, 0) solved by one warp), FP32,
FP64 and FP32 + refinement, Poisson, Helmholtz and the adjoint solve.
"""
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

# (nx, ny, nz, bc, precisions)
CASES = [
    (512, 128, 64, (0, 0, 0, 0, 1, 1), (cs.FP32, cs.FP32_REFINE)),      # 4 full segments of 16 rows
    (256, 256, 300, (0, 0, 1, 1, 2, 1), (cs.FP32, cs.FP32_REFINE)),     # 10 segments of 30 rows (ragged)
    (256, 160, 96, (0, 0, 2, 2, 3, 3), (cs.FP64, cs.FP32)),             # FP64 tiles, wall-node z
    (400, 99, 170, (0, 0, 3, 3, 1, 1), (cs.FP32, cs.FP64)),             # 11 segments of 16 rows, last 10; last mode tile 16 wide
    (1536, 40, 512, (0, 0, 1, 1, 1, 1), (cs.FP32, cs.FP32_REFINE)),     # the bench's duct lines: 16 segments of 32 rows
]


def _solve_all():
    out = {}
    for ci, (nx, ny, nz, bc, modes) in enumerate(CASES):
        plan = cs.channel_plan(nx, ny, nz, beta=1.7, bc=bc)
        f64 = torch.from_numpy(S.gaussian(9300 + ci, (nz, ny, nx))).cuda()
        for mode in modes:
            plan.set_precision(mode, 2)
            f = f64.float() if mode == cs.FP32 else f64
            for alpha in (None, 1e-3):
                for rep in range(2):        # computed, then cached segment-entry pivots
                    u = plan.poisson(f) if alpha is None else plan.helmholtz(alpha, f)
                    torch.cuda.synchronize()
                    out[f"{ci}_{mode}_{alpha}_{rep}"] = u.cpu().numpy()
                if mode != cs.FP32_REFINE:
                    g = plan.poisson_adjoint(f) if alpha is None else plan.helmholtz_adjoint(alpha, f)
                    torch.cuda.synchronize()
                    out[f"{ci}_{mode}_{alpha}_adj"] = g.cpu().numpy()
        assert plan.status() == 0
    return out


def test_persistent_and_one_tile_z_kernels_agree_bitwise(cuda_device, tmp_path):
    mine = _solve_all()
    dst = tmp_path / "persistent.npz"
    code = ("import sys, numpy as np; sys.path.insert(0, %r); "
            "import tests.test_gpu_zpersist as T; np.savez(%r, **T._solve_all())" % (ROOT, str(dst)))
    env = dict(os.environ, CALES_ZPERSIST="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    other = np.load(dst)
    for k, v in mine.items():
        w = other[k]
        ci, mode, alpha = k.split("_")[:3]
        bc = CASES[int(ci)][3]
        singular = all(b in (0, 1) for b in bc)
        if singular and int(mode) == cs.FP32_REFINE and alpha == "None":
            # singular Poisson with refinement: the gauge sum is an FP64 atomic reduction
            assert np.linalg.norm(v - w) <= 1e-13 * np.linalg.norm(w), k
        else:
            assert np.array_equal(v, w), (k, float(np.abs(v - w).max()))
