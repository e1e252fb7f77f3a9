"""GB300 bootstrap algebraic multigrid for the stationary vector of a Markov chain.

The method (Brannick, Kahl, Sokolovic: an adaptively constructed AMG
preconditioner for irreducible Markov chains) runs in ``libbamg.so``: CUDA
kernels for sm_103a behind the C ABI of ``include/bamg.h``.  This package is
the Python binding (``api``) and the in-tree build (``build``).
"""
from .api import (Hierarchy, bamg_params_default, bamg_setup, bamg_solve, bamg_solve_host,
                  bamg_solve_params_default, bamg_vcycle, launch_count)

__all__ = ["Hierarchy", "bamg_params_default", "bamg_setup", "bamg_solve", "bamg_solve_host",
           "bamg_solve_params_default", "bamg_vcycle", "launch_count"]
