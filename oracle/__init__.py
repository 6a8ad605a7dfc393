"""FP64 CPU oracle for the fast Poisson/Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the CUDA library and its Python binding) never imports, links
or executes anything here, and this package imports nothing from the product.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed-form discrete eigenfunctions, dense LU,
second-order convergence of the stencil, residuals, transpose identities,
finite differences).  No function is "parity unpinned".
"""
from .cales_oracle import *  # noqa: F401,F403
from .closure_oracle import *  # noqa: F401,F403
from .sgs_oracle import *  # noqa: F401,F403
from .rk3_oracle import *  # noqa: F401,F403
