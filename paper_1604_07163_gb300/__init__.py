"""GB300-native geometric-multigrid-preconditioned CG for -div(k grad phi) = f.

The compute path is the CUDA library ``libmgpcg.so`` (C ABI in include/mg.h);
this package is its Python binding.  Every solver object loads the library
and raises ImportError when it has not been built
(``python -m paper_1604_07163_gb300.build``); there is no CPU fallback.
"""
from ._lib import EXPORTS, MgError
from .solver import MGSolveFn, MGSolver, Params, Stats, mg_solve

__all__ = ["MGSolver", "MGSolveFn", "Params", "Stats", "MgError", "mg_solve", "EXPORTS"]
