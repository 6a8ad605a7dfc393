"""The compile-time-size transform kernels against the run-time-size ones.

Both variants run the same radix passes with the same twiddles in the same
order, so their solves agree bit for bit.  The run-time-size kernels run in a
child process started with CALES_STATIC_FFT=0 (the switch is read once per
process).  Sizes: every specialised length (periodic rows n = 256, 512, 1536;
columns n = 128, 256, 512 with every kind), FP32 and FP32 + refinement.
"""
import json
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

# (nx, ny, nz, bc): x periodic rows of the specialised lengths, y of each kind
CASES = [
    (256, 128, 24, (0, 0, 0, 0, 1, 1)),
    (512, 256, 20, (0, 0, 1, 1, 1, 1)),
    (1536, 512, 8, (0, 0, 2, 2, 2, 1)),
    (512, 128, 16, (0, 0, 2, 2, 1, 1)),
    (64, 512, 6, (0, 0, 0, 0, 1, 1)),      # y n = 512 periodic: the one-buffer column kernel
    (96, 512, 5, (0, 0, 1, 1, 1, 1)),      # y n = 512 cosine
    (40, 512, 4, (0, 0, 2, 2, 2, 2)),      # y n = 512 sine, a partial 16-column tile
]
MODES = [cs.FP32, cs.FP32_REFINE]


def _solve_all():
    out = {}
    for ci, (nx, ny, nz, bc) in enumerate(CASES):
        plan = cs.channel_plan(nx, ny, nz, beta=1.6, bc=bc)
        f64 = torch.from_numpy(S.gaussian(9100 + ci, (nz, ny, nx))).cuda()
        for mode in MODES:
            plan.set_precision(mode, 2)
            f = f64.float() if mode == cs.FP32 else f64
            for alpha in (None, 1e-3):
                u = plan.poisson(f) if alpha is None else plan.helmholtz(alpha, f)
                torch.cuda.synchronize()
                out[f"{ci}_{mode}_{alpha}"] = u.cpu().numpy()
        assert plan.status() == 0
    return out


def test_static_and_runtime_size_kernels_agree_bitwise(cuda_device, tmp_path):
    mine = _solve_all()
    dst = tmp_path / "runtime_size.npz"
    code = ("import sys, numpy as np; sys.path.insert(0, %r); "
            "import tests.test_gpu_static_fft as T; np.savez(%r, **T._solve_all())" % (ROOT, str(dst)))
    env = dict(os.environ, CALES_STATIC_FFT="0")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    other = np.load(dst)
    for k, v in mine.items():
        w = other[k]
        ci, mode, alpha = k.split("_")
        bc = CASES[int(ci)][3]
        singular = all(b in (0, 1) for b in bc)
        if singular and int(mode) == cs.FP32_REFINE and alpha == "None":
            # singular Poisson with refinement: the gauge sum is an FP64 atomic reduction
            assert np.linalg.norm(v - w) <= 1e-13 * np.linalg.norm(w), k
        else:
            assert np.array_equal(v, w), (k, float(np.abs(v - w).max()))
