"""GB300 cut-cell multigrid: a fourth-order finite-volume solver for
a u_xx + b u_xy + c u_yy = f on a box minus elliptic holes (arXiv 2601.02975).

The solver runs in libccmg.so (CUDA, sm_103a) behind the C ABI of
include/ccmg.h; `Hierarchy` is its Python binding.
"""
from ._lib import (CYCLE_FMG, CYCLE_V, CYCLE_W, PREC_FP64, PREC_MIXED, SMOOTHER_JACOBI,
                   SMOOTHER_MCGS, CCError, Hierarchy, cache_clear, default_options, lib,
                   serve_budget, solve_batch)

__all__ = ["Hierarchy", "CCError", "default_options", "lib", "solve_batch", "serve_budget",
           "cache_clear", "CYCLE_V", "CYCLE_W",
           "CYCLE_FMG", "PREC_FP64", "PREC_MIXED", "SMOOTHER_JACOBI", "SMOOTHER_MCGS"]
