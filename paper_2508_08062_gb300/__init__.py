"""GB300-native (sm_103a) AA-PDHG / FAA-PDHG solver for linear programs (arXiv 2508.08062).

The solver lives in the CUDA library ``libaapdhg.so`` (C ABI: ``include/aapdhg.h``);
``binding`` is a thin ctypes wrapper over it.  Build with ``build.build()``.
"""
from .binding import (AA, FAA, FP64, MIXED, PDHG, AAPDHGError, BatchSolver, Server,  # noqa: F401
                      Solver, load, use_torch_allocator)
