"""GB300 (sm_103a) implementation of the HPR-QP iteration (arXiv 2507.02470).

The solver runs in the CUDA library ``libhprqp.so`` behind the C ABI of include/hprqp.h;
this package holds its sources (``csrc/``), the build step (``build``) and a thin ctypes
binding (``Solver`` and the raw ``lib()`` entry points).
"""
from .build import build  # noqa: F401
from ._lib import (BatchSolver, HPRQPError, Solver, default_params, fp64_rate, lib, lib_path,  # noqa: F401
                   STATUS_NAMES)

__all__ = ["build", "Solver", "BatchSolver", "HPRQPError", "default_params", "fp64_rate", "lib", "lib_path",
           "STATUS_NAMES"]
