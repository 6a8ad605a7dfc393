"""The C-ABI library builds, loads and exports every symbol that
include/*.h declares; argument validation runs without a GPU."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2411_09364_gb300 import build, _native
    build.build()
    return _native.lib()


def declared_functions():
    names = []
    for h in sorted((ROOT / "include").glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(cales_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cales_plan", "cales_poisson_solve", "cales_helmholtz_solve", "cales_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_invalid_plans_are_rejected_on_host(lib):
    bc = (C.c_int * 6)(0, 0, 0, 0, 1, 1)
    dzc = np.ones(9)
    dzf = np.ones(8)
    h = C.c_void_p()
    dp = C.POINTER(C.c_double)
    args = lambda nx, ny, nz, b=bc, dx=1.0: lib.cales_plan(C.byref(h), nx, ny, nz, b, dx, 1.0,
                                                            dzc.ctypes.data_as(dp), dzf.ctypes.data_as(dp))
    assert args(0, 4, 8) == -1                     # empty grid
    assert args(4, 4, 8, dx=-1.0) == -1            # bad spacing
    assert args(4, 4, 8, (C.c_int * 6)(0, 1, 0, 0, 1, 1)) == -1    # periodic paired with a wall
    assert args(4, 4, 8, (C.c_int * 6)(1, 3, 0, 0, 1, 1)) == -2    # a wall node beside a Neumann face
    assert args(6, 4, 8, (C.c_int * 6)(3, 3, 0, 0, 1, 1)) == -2    # node unknowns: n + 1 = 7 has no FFT here
    assert args(5, 4, 8, (C.c_int * 6)(1, 2, 0, 0, 1, 1)) == -2    # mixed sides need an even n
    assert args(4, 4, 2, (C.c_int * 6)(0, 0, 0, 0, 0, 0)) == -2    # periodic z needs three cells
    assert args(4, 4, 8, (C.c_int * 6)(0, 0, 0, 0, 0, 1)) == -1    # periodic z on one side only
    wrap = np.ones(9)
    wrap[8] = 1.5                                  # periodic z: dzc[0] and dzc[nz] disagree
    assert lib.cales_plan(C.byref(h), 4, 4, 8, (C.c_int * 6)(0, 0, 0, 0, 0, 0), 1.0, 1.0,
                          wrap.ctypes.data_as(dp), dzf.ctypes.data_as(dp)) == -1
    bad = np.ones(9)
    bad[3] = 0.0
    assert lib.cales_plan(C.byref(h), 4, 4, 8, bc, 1.0, 1.0, bad.ctypes.data_as(dp), dzf.ctypes.data_as(dp)) == -1
    assert lib.cales_poisson_solve(None, None, None, None) == -1
    assert lib.cales_set_precision(None, 0, 2) == -1
    assert lib.cales_strerror(-2) == b"unsupported size or boundary combination"


def test_next_row_entries_reject_null_plans_on_host(lib):
    """The closure and substep entries check their plan before any device work."""
    d = C.c_double
    assert lib.cales_eddy_viscosity(None, d(0.1), d(1e-3), d(0.05), None, None, None, None, None) == -1
    assert lib.cales_rk3_substep(None, 0, d(1e-3), d(1e-3), d(0.1), d(0.05), *([None] * 10)) == -1
    assert lib.cales_rk3_substep_cn(None, None, None, 1, 0, d(1e-3), d(1e-3), d(0.1), d(0.05),
                                    *([None] * 10)) == -1
    assert lib.cales_helmholtz_z_solve(None, d(1e-3), None, None, None) == -1
