"""GPU-native exact solver for the feasibility market split problem.

The work runs in ``libmsp.so`` (hand-written sm_103a CUDA kernels behind the
C ABI of ``include/msp.h``); this package only marshals arguments through
ctypes.  See :mod:`paper_2507_05045_gb300.msp` for the Python API.
"""
from .msp import (MspError, Instance, Server, solve_all, solve_batch, lib_path,  # noqa: F401
                  load_library, solve_small_noalloc, plan_info, EXPORTED_SYMBOLS)
