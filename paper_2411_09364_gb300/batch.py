"""Batched Runge-Kutta-substep solves through the C ABI (cales_batch_*).

One substep of the fractional-step method (Algorithm 1, Sec. 2.2) with
Crank-Nicolson viscous terms needs, per domain, three Helmholtz solves
(Eq. 18) for u, v, w and one Poisson solve (Eq. 12).  On a channel domain
(periodic x, y; walls in z) u and v are cell-centred in z (Dirichlet walls,
ghost = -interior), w lives on the z-faces (Dirichlet at the wall nodes,
nz-1 unknowns) and p is cell-centred with Neumann walls.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _native as N
from .solver import FP32_REFINE, Plan, _stream, cell_spacings, face_spacings, tanh_faces


class Batch:
    """A list of (plan, kind, alpha) solves executed as one fork/join, optionally
    captured once into a CUDA graph."""

    def __init__(self, plans, kinds, alphas):
        n = len(plans)
        self.plans = list(plans)
        arr = (C.c_void_p * n)(*[p.handle.value for p in plans])
        ks = (C.c_int * n)(*[int(k) for k in kinds])
        al = (C.c_double * n)(*[float(a) for a in alphas])
        h = C.c_void_p()
        N.check(N.lib().cales_batch_create(C.byref(h), n, arr, ks, al), "cales_batch_create")
        self._h = h
        self.kinds = list(kinds)
        self.alphas = list(alphas)
        self._keep = None

    @staticmethod
    def _ptrs(ts):
        return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def solve(self, fs, us, stream=None):
        N.check(N.lib().cales_batch_solve(self._h, self._ptrs(fs), self._ptrs(us), _stream(stream)),
                "cales_batch_solve")

    def capture(self, fs, us, stream=None):
        """Record the batch for these buffers into one CUDA graph (needs a non-default stream)."""
        st = stream if stream is not None else torch.cuda.Stream()
        self._keep = (list(fs), list(us), st)
        N.check(N.lib().cales_batch_capture(self._h, self._ptrs(fs), self._ptrs(us), _stream(st)),
                "cales_batch_capture")
        return st

    def launch(self, stream=None):
        N.check(N.lib().cales_batch_launch(self._h, _stream(stream)), "cales_batch_launch")

    def set_grouped(self, on: bool = True):
        """Grouped stage launches (default) or the fork/join over streams."""
        N.check(N.lib().cales_batch_set_grouped(self._h, 1 if on else 0), "cales_batch_set_grouped")
        return self

    def grouped(self) -> bool:
        """Whether the last solve or capture used the grouped stage launches."""
        v = C.c_int(0)
        N.check(N.lib().cales_batch_grouped(self._h, C.byref(v)), "cales_batch_grouped")
        return bool(v.value)

    def graph_nodes(self) -> int:
        n = C.c_ulong(0)
        N.check(N.lib().cales_batch_graph_nodes(self._h, C.byref(n)), "cales_batch_graph_nodes")
        return n.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().cales_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def channel_domain_plans(nx, ny, nz, beta=1.8, lx=2 * math.pi, ly=math.pi, lz=2.0, precision=FP32_REFINE,
                         sweeps=2):
    """Plans of one channel domain: (u and v: z Dirichlet walls, w: wall nodes, p: Neumann)."""
    zf = tanh_faces(nz, beta, lz)
    dzc, dzf = cell_spacings(zf)
    wdzc, wdzf = face_spacings(zf)
    dx, dy = lx / nx, ly / ny
    uv = Plan(nx, ny, nz, (0, 0, 0, 0, 2, 2), dx, dy, dzc, dzf, precision, sweeps)
    u2 = Plan(nx, ny, nz, (0, 0, 0, 0, 2, 2), dx, dy, dzc, dzf, precision, sweeps)
    w = Plan(nx, ny, nz - 1, (0, 0, 0, 0, 3, 3), dx, dy, wdzc, wdzf, precision, sweeps)
    p = Plan(nx, ny, nz, (0, 0, 0, 0, 1, 1), dx, dy, dzc, dzf, precision, sweeps)
    return {"u": uv, "v": u2, "w": w, "p": p}


def rk3_substep_batch(domains, alphas, precision=FP32_REFINE, sweeps=2, beta=1.8, autotune=True, cache_path=None):
    """Plans and solve list of one RK3 substep over several channel domains.

    domains: list of (nx, ny, nz); alphas: Helmholtz alpha per domain.  With
    ``autotune`` every plan's launch schedule comes from the device autotuner
    (cales_autotune; looked up in / stored to the JSON ``cache_path`` when
    given), before the batch is built.
    Returns (batch, plan list, [(domain index, field name)] in batch order).
    """
    plans, kinds, als, tags = [], [], [], []
    for d, (nx, ny, nz) in enumerate(domains):
        dp = channel_domain_plans(nx, ny, nz, beta=beta, precision=precision, sweeps=sweeps)
        if autotune:
            for pl in dp.values():
                pl.autotune(cache_path)
        for name in ("u", "v", "w", "p"):
            plans.append(dp[name])
            kinds.append(0 if name == "p" else 1)
            als.append(0.0 if name == "p" else alphas[d])
            tags.append((d, name))
    return Batch(plans, kinds, als), plans, tags
