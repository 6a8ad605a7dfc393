"""ctypes declarations of the C ABI in include/cales.h (argument marshalling only).

The library is the in-tree ``_build/libcales.so`` produced by ``build.py``.
There is no fallback: if the library is missing or does not load, every
entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libcales.so"
_lib = None

vp = C.c_void_p
ip = C.POINTER(C.c_int)
dp = C.POINTER(C.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "cales_plan": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int, C.c_int, ip, C.c_double, C.c_double, dp, dp]),
    "cales_set_precision": (C.c_int, [vp, C.c_int, C.c_int]),
    "cales_poisson_solve": (C.c_int, [vp, vp, vp, vp]),
    "cales_helmholtz_solve": (C.c_int, [vp, C.c_double, vp, vp, vp]),
    "cales_helmholtz_z_solve": (C.c_int, [vp, C.c_double, vp, vp, vp]),
    "cales_eddy_viscosity": (C.c_int, [vp, C.c_double, C.c_double, C.c_double, vp, vp, vp, vp, vp]),
    "cales_rk3_substep": (C.c_int, [vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, vp, vp, vp, vp, vp,
                                    vp, vp, vp, vp, vp]),
    "cales_rk3_substep_cn": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                       vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "cales_poisson_solve_adjoint": (C.c_int, [vp, vp, vp, vp]),
    "cales_poisson_solve_noalloc": (C.c_int, [vp, vp, vp, vp]),
    "cales_helmholtz_solve_adjoint": (C.c_int, [vp, C.c_double, vp, vp, vp]),
    "cales_residual": (C.c_int, [vp, C.c_double, vp, vp, vp, vp]),
    "cales_get_status": (C.c_int, [vp, ip]),
    "cales_strerror": (C.c_char_p, [C.c_int]),
    "cales_destroy": (None, [vp]),
    "cales_profile_enable": (C.c_int, [vp, C.c_int]),
    "cales_divergence": (C.c_int, [vp, vp, vp, vp, vp, vp]),
    "cales_gradient": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "cales_divergence_adjoint": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "cales_zero": (C.c_int, [vp, C.c_ulong, vp]),
    "cales_set_schedule": (C.c_int, [vp, ip]),
    "cales_get_schedule": (C.c_int, [vp, ip]),
    "cales_autotune": (C.c_int, [vp, C.c_char_p, vp]),
    "cales_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(vp), ip, dp]),
    "cales_batch_solve": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), vp]),
    "cales_batch_capture": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), vp]),
    "cales_batch_launch": (C.c_int, [vp, vp]),
    "cales_batch_graph_nodes": (C.c_int, [vp, C.POINTER(C.c_ulong)]),
    "cales_batch_set_grouped": (C.c_int, [vp, C.c_int]),
    "cales_batch_grouped": (C.c_int, [vp, ip]),
    "cales_batch_destroy": (None, [vp]),
    "cales_gradient_adjoint": (C.c_int, [vp, vp, vp, vp, vp, vp]),
    "cales_stencil27": (C.c_int, [vp, vp, C.c_float, C.c_float, C.POINTER(vp), C.POINTER(vp), vp]),
    "cales_stencil27_weight_grad": (C.c_int, [vp, C.POINTER(vp), C.POINTER(vp), vp, vp]),
    "cales_sq_error": (C.c_int, [C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_long), C.c_float, vp, vp]),
    "cales_adam_step": (C.c_int, [vp, vp, vp, vp, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                                  C.c_float, vp]),
    "cales_profile_read": (C.c_int, [vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_float)]),
}


def library_path() -> Path:
    return Path(os.environ.get("CALES_LIB", _LIB_PATH))


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not path.exists():
            raise RuntimeError(f"CUDA library {path} is missing: run paper_2411_09364_gb300/build.py "
                               "(or __graft_entry__.build()) first")
        handle = C.CDLL(str(path))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


class CalesError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().cales_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != 0:
        raise CalesError(code, where)
