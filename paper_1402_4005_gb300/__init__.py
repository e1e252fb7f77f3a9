"""GB300 bootstrap algebraic multigrid for the stationary vector of a Markov chain.

The method (Brannick, Kahl, Sokolovic: an adaptively constructed AMG
preconditioner for irreducible Markov chains) runs in ``libbamg.so``: CUDA
kernels for sm_103a behind the C ABI of ``include/bamg.h``.  This package is
the Python binding (``api``) and the in-tree build (``build``).
"""
from .api import (Batch, Hierarchy, bamg_mlp_forward, bamg_mlp_grad, bamg_mlp_harvest, bamg_mlp_init,
                  bamg_mlp_load, bamg_mlp_num_params, bamg_mlp_save, bamg_mlp_train, bamg_params_default, bamg_setup, bamg_setup_batched,
                  bamg_setup_judged, bamg_solve, bamg_solve_batched, bamg_solve_host, bamg_solve_params_default,
                  bamg_vcycle, bamg_vcycle_batched, bamg_vcycle_factor, launch_count)

__all__ = ["Batch", "Hierarchy", "bamg_mlp_forward", "bamg_mlp_grad", "bamg_mlp_harvest", "bamg_mlp_init",
           "bamg_mlp_load", "bamg_mlp_num_params", "bamg_mlp_save", "bamg_mlp_train", "bamg_params_default", "bamg_setup", "bamg_setup_batched",
           "bamg_setup_judged", "bamg_solve", "bamg_solve_batched", "bamg_solve_host",
           "bamg_solve_params_default", "bamg_vcycle", "bamg_vcycle_batched", "bamg_vcycle_factor",
           "launch_count"]
