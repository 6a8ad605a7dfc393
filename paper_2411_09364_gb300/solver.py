"""Python face of the C ABI: the same entry points as include/cales.h, taking
torch tensors (device memory) and the current torch CUDA stream.

Only argument marshalling happens here; every step of a solve runs in the
library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _native as N

BC_P, BC_N, BC_D, BC_DF = 0, 1, 2, 3
FP64, FP32, FP32_REFINE, FP32_REFINE_FAST = 0, 1, 2, 3
SCHED_LEN = 6          # CALES_SCHED_LEN: launch schedule entries
_DTYPE = {FP64: torch.float64, FP32: torch.float32, FP32_REFINE: torch.float64, FP32_REFINE_FAST: torch.float64}


def cell_spacings(zf):
    """dzc[0..nz], dzf[0..nz-1] of cell-centred unknowns from faces zf[0..nz]
    (boundary entries of dzc: mirror distance = width of the wall cell)."""
    zf = np.asarray(zf, dtype=np.float64)
    dzf = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzc = np.concatenate([[dzf[0]], np.diff(zc), [dzf[-1]]])
    return dzc, dzf


def face_spacings(zf):
    """dzc, dzf of node-centred unknowns on the interior faces zf[1..nz-1]."""
    zf = np.asarray(zf, dtype=np.float64)
    zc = 0.5 * (zf[1:] + zf[:-1])
    return np.diff(zf), np.diff(zc)


def channel_velocity_plans(nx, ny, zf, dx, dy, precision=None, sweeps=2):
    """(uv_plan, w_plan) of a channel with faces zf[0..nz]: u and v cell-centred
    with Dirichlet z walls, w on the interior faces with wall nodes."""
    dzc, dzf = cell_spacings(zf)
    wdzc, wdzf = face_spacings(zf)
    nz = len(zf) - 1
    prec = FP64 if precision is None else precision
    uv = Plan(nx, ny, nz, (0, 0, 0, 0, 2, 2), dx, dy, dzc, dzf, prec, sweeps)
    w = Plan(nx, ny, nz - 1, (0, 0, 0, 0, 3, 3), dx, dy, wdzc, wdzf, prec, sweeps)
    return uv, w


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor, dtype, numel: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be contiguous with {numel} elements")
    return t.data_ptr()


class Plan:
    """Owns a cales_plan_t (see cales_plan in include/cales.h)."""

    def __init__(self, nx, ny, nz, bc, dx, dy, dzc, dzf, precision=FP64, sweeps=2):
        dzc = np.ascontiguousarray(dzc, dtype=np.float64)
        dzf = np.ascontiguousarray(dzf, dtype=np.float64)
        if dzc.shape != (nz + 1,) or dzf.shape != (nz,):
            raise ValueError("dzc must have nz+1 and dzf nz entries")
        bcs = (C.c_int * 6)(*[int(b) for b in bc])
        h = C.c_void_p()
        N.check(N.lib().cales_plan(C.byref(h), int(nx), int(ny), int(nz), bcs, float(dx), float(dy),
                                   dzc.ctypes.data_as(N.dp), dzf.ctypes.data_as(N.dp)), "cales_plan")
        self._h = h
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.bc = tuple(int(b) for b in bc)
        self.dx, self.dy = float(dx), float(dy)
        self.dzc, self.dzf = dzc, dzf
        self.precision = FP64
        self.sweeps = sweeps
        self.set_precision(precision, sweeps)

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def numel(self):
        return self.nx * self.ny * self.nz

    @property
    def dtype(self):
        return _DTYPE[self.precision]

    def set_precision(self, mode: int, sweeps: int = 2):
        N.check(N.lib().cales_set_precision(self._h, int(mode), int(sweeps)), "cales_set_precision")
        self.precision, self.sweeps = int(mode), int(sweeps)
        return self

    def _io(self, f, out):
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=f.device)
        return (_ptr(f, self.dtype, self.numel, "f"), _ptr(out, self.dtype, self.numel, "out"), out)

    def poisson(self, f, out=None, stream=None):
        pf, po, out = self._io(f, out)
        N.check(N.lib().cales_poisson_solve(self._h, pf, po, _stream(stream)), "cales_poisson_solve")
        return out

    def helmholtz(self, alpha, f, out=None, stream=None):
        pf, po, out = self._io(f, out)
        N.check(N.lib().cales_helmholtz_solve(self._h, float(alpha), pf, po, _stream(stream)),
                "cales_helmholtz_solve")
        return out

    def helmholtz_z(self, alpha, f, out=None, stream=None):
        """(I - alpha L_z) u = f on every (i, j) line (wall-normal implicit step, Eq. 21)."""
        pf, po, out = self._io(f, out)
        N.check(N.lib().cales_helmholtz_z_solve(self._h, float(alpha), pf, po, _stream(stream)),
                "cales_helmholtz_z_solve")
        return out

    def eddy_viscosity(self, cs, nu, utau, u, v, w, out=None, stream=None):
        """Smagorinsky / van Driest eddy viscosity at the cell centres (Eq. 4)."""
        n = self.numel
        nw = self.nx * self.ny * (self.nz + 1)
        pu, pv = _ptr(u, self.dtype, n, "u"), _ptr(v, self.dtype, n, "v")
        pw = _ptr(w, self.dtype, nw, "w")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=u.device)
        po = _ptr(out, self.dtype, n, "out")
        N.check(N.lib().cales_eddy_viscosity(self._h, float(cs), float(nu), float(utau), pu, pv, pw, po,
                                             _stream(stream)), "cales_eddy_viscosity")
        return out

    def rk3_work(self, device="cuda"):
        """Scratch for rk3_substep: 3 nx ny nz + nx ny (nz + 1) elements."""
        return torch.empty(3 * self.numel + self.nx * self.ny * (self.nz + 1), dtype=self.dtype, device=device)

    def rk3_substep(self, stage, dt, nu, cs, utau, u, v, w, p, nut, ru, rv, rw, work=None, stream=None):
        """One explicit RK3 pressure-correction substep (Eqs. 11-14, then Eq. 4),
        in place: (u, v, w, p, nut) advance to stage + 1 and (ru, rv, rw) hold
        R^k for the next stage (their input is R^{k-1}, unread at stage 0)."""
        n = self.numel
        nw = self.nx * self.ny * (self.nz + 1)
        if work is None:
            work = self.rk3_work(u.device)
        ptrs = [_ptr(t, self.dtype, m, name) for t, m, name in
                ((u, n, "u"), (v, n, "v"), (w, nw, "w"), (p, n, "p"), (nut, n, "nut"), (ru, n, "ru"),
                 (rv, n, "rv"), (rw, nw, "rw"), (work, 3 * n + nw, "work"))]
        N.check(N.lib().cales_rk3_substep(self._h, int(stage), float(dt), float(nu), float(cs), float(utau), *ptrs,
                                          _stream(stream)), "cales_rk3_substep")
        return work

    def rk3_substep_cn(self, uv_plan, w_plan, implicit, stage, dt, nu, cs, utau, u, v, w, p, nut, ru, rv, rw,
                       work=None, stream=None):
        """One Crank-Nicolson RK3 substep in place: implicit = 1 (Eqs. 17-19,
        Helmholtz solves on uv_plan / w_plan) or 2 (Eqs. 20-22, line solves);
        see channel_velocity_plans for the two velocity plans."""
        n = self.numel
        nw = self.nx * self.ny * (self.nz + 1)
        if work is None:
            work = self.rk3_work(u.device)
        ptrs = [_ptr(t, self.dtype, m, name) for t, m, name in
                ((u, n, "u"), (v, n, "v"), (w, nw, "w"), (p, n, "p"), (nut, n, "nut"), (ru, n, "ru"),
                 (rv, n, "rv"), (rw, nw, "rw"), (work, 3 * n + nw, "work"))]
        N.check(N.lib().cales_rk3_substep_cn(self._h, uv_plan._h, w_plan._h, int(implicit), int(stage), float(dt),
                                             float(nu), float(cs), float(utau), *ptrs, _stream(stream)),
                "cales_rk3_substep_cn")
        return work

    def poisson_adjoint(self, w, out=None, stream=None):
        pf, po, out = self._io(w, out)
        N.check(N.lib().cales_poisson_solve_adjoint(self._h, pf, po, _stream(stream)),
                "cales_poisson_solve_adjoint")
        return out

    def helmholtz_adjoint(self, alpha, w, out=None, stream=None):
        pf, po, out = self._io(w, out)
        N.check(N.lib().cales_helmholtz_solve_adjoint(self._h, float(alpha), pf, po, _stream(stream)),
                "cales_helmholtz_solve_adjoint")
        return out

    def residual(self, u, f, alpha=None, out=None, stream=None):
        """FP64 r = f - L u (alpha None) or f - (I - alpha L) u."""
        n = self.numel
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device=u.device)
        N.check(N.lib().cales_residual(self._h, -1.0 if alpha is None else float(alpha),
                                       _ptr(u, torch.float64, n, "u"), _ptr(f, torch.float64, n, "f"),
                                       _ptr(out, torch.float64, n, "out"), _stream(stream)), "cales_residual")
        return out

    def set_schedule(self, sched):
        """{x budget KB, y tile, z warps, z segment rows, FFT radix order, z variant};
        shorter lists are padded with 0 (the heuristic)."""
        vals = [int(v) for v in sched] + [0] * (SCHED_LEN - len(sched))
        arr = (C.c_int * SCHED_LEN)(*vals[:SCHED_LEN])
        N.check(N.lib().cales_set_schedule(self._h, arr), "cales_set_schedule")

    def schedule(self):
        arr = (C.c_int * SCHED_LEN)()
        N.check(N.lib().cales_get_schedule(self._h, arr), "cales_get_schedule")
        return tuple(arr)

    def autotune(self, cache_path=None, stream=None):
        """Time candidate schedules on the device (or read them from the JSON cache)."""
        path = None if cache_path is None else str(cache_path).encode()
        N.check(N.lib().cales_autotune(self._h, path, _stream(stream)), "cales_autotune")
        return self.schedule()

    def status(self) -> int:
        v = C.c_int(0)
        N.check(N.lib().cales_get_status(self._h, C.byref(v)), "cales_get_status")
        return v.value

    def profile(self, on: bool = True):
        N.check(N.lib().cales_profile_enable(self._h, 1 if on else 0), "cales_profile_enable")

    def profile_read(self):
        names = (C.c_char_p * 4096)()
        ms = (C.c_float * 4096)()
        n = N.lib().cales_profile_read(self._h, 4096, names, ms)
        return [(names[i].decode(), float(ms[i])) for i in range(max(n, 0))]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            N.lib().cales_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# C-ABI names (same arguments as include/cales.h, tensors in place of pointers)
def cales_plan(nx, ny, nz, bc, dx, dy, dzc, dzf) -> Plan:
    return Plan(nx, ny, nz, bc, dx, dy, dzc, dzf)


def cales_set_precision(plan: Plan, mode: int, sweeps: int = 2) -> None:
    plan.set_precision(mode, sweeps)


def cales_poisson_solve(plan: Plan, f, p, stream=None):
    return plan.poisson(f, p, stream)


def cales_helmholtz_solve(plan: Plan, alpha, f, u, stream=None):
    return plan.helmholtz(alpha, f, u, stream)


def cales_helmholtz_z_solve(plan: Plan, alpha, f, u, stream=None):
    plan.helmholtz_z(alpha, f, u, stream)


def cales_poisson_solve_adjoint(plan: Plan, w, g, stream=None):
    return plan.poisson_adjoint(w, g, stream)


def cales_helmholtz_solve_adjoint(plan: Plan, alpha, w, g, stream=None):
    return plan.helmholtz_adjoint(alpha, w, g, stream)


def cales_residual(plan: Plan, alpha, u, f, r, stream=None):
    return plan.residual(u, f, None if alpha is None or alpha < 0 else alpha, r, stream)


def cales_get_status(plan: Plan) -> int:
    return plan.status()


def cales_destroy(plan: Plan) -> None:
    plan.close()


def tanh_faces(nz: int, beta: float, lz: float = 2.0) -> np.ndarray:
    """Wall-normal faces z_k = lz/2 (1 + tanh(beta (2k/nz - 1)) / tanh(beta)), k = 0..nz,
    of a channel or duct clustered at both walls; beta <= 0 gives a uniform grid."""
    k = np.arange(nz + 1, dtype=np.float64)
    if beta <= 0:
        return lz * k / nz
    return 0.5 * lz * (1.0 + np.tanh(beta * (2.0 * k / nz - 1.0)) / math.tanh(beta))


def channel_plan(nx, ny, nz, beta=1.8, lx=2 * math.pi, ly=math.pi, lz=2.0, bc=(0, 0, 0, 0, 1, 1),
                 precision=FP64, sweeps=2, faces=None):
    """Plan on a tanh-stretched channel grid (cell-centred unknowns in z)."""
    if faces is None:
        faces = tanh_faces(nz, beta, lz)
    dzc, dzf = cell_spacings(faces)
    return Plan(nx, ny, nz, bc, lx / nx, ly / ny, dzc, dzf, precision, sweeps)
