"""GB300-native fast direct solver for the pressure Poisson and Crank-Nicolson
velocity Helmholtz equations on a staggered grid (eigenfunction expansion:
FFT/DCT/DST in x, y; Thomas per mode in z).

The compute path is the CUDA library in ``csrc/`` (C ABI: include/cales.h);
``solver`` marshals torch tensors into it.
"""
from .solver import (BC_D, BC_DF, BC_N, BC_P, FP32, FP32_REFINE, FP64, Plan, cales_destroy,
                     cales_get_status, cales_helmholtz_solve, cales_helmholtz_solve_adjoint, cales_plan,
                     cales_poisson_solve, cales_poisson_solve_adjoint, cales_residual, cales_set_precision,
                     cell_spacings, channel_plan, face_spacings)

__all__ = [n for n in dir() if not n.startswith("_")]
