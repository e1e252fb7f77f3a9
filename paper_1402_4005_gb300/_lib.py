"""ctypes declarations of the C ABI in include/bamg.h and include/bamg_steps.h.

Loads ``_build/libbamg.so`` (built in-tree by ``build.py``).  There is no
fallback: if the library is missing or fails to load, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbamg.so")

STATUS = {0: "BAMG_OK", 1: "BAMG_ERR_ARG", 2: "BAMG_ERR_NOT_STOCHASTIC", 3: "BAMG_ERR_CUDA",
          4: "BAMG_ERR_OOM", 5: "BAMG_ERR_NOT_CONVERGED", 6: "BAMG_ERR_BREAKDOWN",
          7: "BAMG_ERR_NUMERIC", 8: "BAMG_ERR_TIMEOUT", 9: "BAMG_ERR_UNSUPPORTED",
          10: "BAMG_ERR_IO"}

vp = C.c_void_p
i32 = C.c_int
i64 = C.c_int64
f64 = C.c_double
u64 = C.c_uint64
dp = C.POINTER(C.c_double)
i64p = C.POINTER(C.c_int64)
ip = C.POINTER(C.c_int)


class Csr(C.Structure):
    _fields_ = [("n", i64), ("nnz", i64), ("row_ptr", vp), ("col_idx", vp), ("val", vp),
                ("on_device", i32), ("nx", i32), ("ny", i32)]


class Params(C.Structure):
    _fields_ = [("r", i32), ("max_levels", i32), ("coarse_min", i32), ("nu_setup", i32),
                ("nu_pre", i32), ("nu_post", i32), ("c_min", i32), ("c_max", i32),
                ("omega", f64), ("coarsening", i32), ("precision", i32), ("restriction", i32),
                ("seed", u64), ("stochastic_tol", f64), ("max_coarse_dense", i32),
                ("interp", i32), ("mlp_params", vp), ("setup_cycles", i32), ("smoother", i32),
                ("ls_ridge", f64)]


class SolveParams(C.Structure):
    _fields_ = [("restart", i32), ("max_iter", i32), ("tol", f64), ("plain", i32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", i32), ("iters_to_1e7", i32), ("levels", i32),
                ("rel_res_1", f64), ("setup_ms", f64), ("solve_ms", f64),
                ("op_cplx", f64), ("grid_cplx", f64), ("min_x", f64), ("fallback_iterations", i32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class CsrView(C.Structure):
    _fields_ = [("rows", i32), ("cols", i32), ("nnz", i32), ("row_ptr", vp), ("col", vp), ("val", vp)]


class LevelView(C.Structure):
    _fields_ = [("n", i32), ("B", CsrView), ("M", CsrView), ("N", CsrView), ("P", CsrView),
                ("Qt", CsrView), ("Q", CsrView), ("cf", vp), ("cmap", vp), ("s", vp), ("t", vp),
                ("jacobi_l1_rows", i32), ("colour", vp), ("ncolours", i32)]


# name -> (restype, argtypes)
SIGNATURES = {
    "bamg_params_default": (i32, [C.POINTER(Params)]),
    "bamg_solve_params_default": (i32, [C.POINTER(SolveParams)]),
    "bamg_setup": (i32, [C.POINTER(Csr), C.POINTER(Params), vp, C.POINTER(vp)]),
    "bamg_vcycle": (i32, [vp, vp, vp, vp]),
    "bamg_solve": (i32, [vp, vp, C.POINTER(SolveParams), C.POINTER(SolveInfo), vp]),
    "bamg_solve_host": (i32, [C.POINTER(Csr), C.POINTER(Params), C.POINTER(SolveParams), dp,
                              C.POINTER(SolveInfo), vp]),
    "bamg_destroy": (None, [vp]),
    "bamg_status_string": (C.c_char_p, [i32]),
    "bamg_last_error": (C.c_char_p, []),
    "bamg_launch_count": (u64, []),
    "bamg_setup_batched": (i32, [C.POINTER(Csr), i32, C.POINTER(Params), i32, vp, C.POINTER(vp)]),
    "bamg_solve_batched": (i32, [vp, vp, C.POINTER(SolveParams), vp, vp]),
    "bamg_vcycle_batched": (i32, [vp, vp, vp, vp]),
    "bamg_batch_offsets": (i32, [vp, i64p]),
    "bamg_batch_lanes": (i32, [vp, i32, ip, ip, ip]),
    "bamg_batch_chain": (vp, [vp, i32]),
    "bamg_destroy_batched": (None, [vp]),
    "bamg_mlp_num_params": (i32, []),
    "bamg_mlp_init": (i32, [vp, u64, vp]),
    "bamg_mlp_save": (i32, [C.c_char_p, vp, i32, vp]),
    "bamg_mlp_load": (i32, [C.c_char_p, vp, i32, vp]),
    "bamg_mlp_forward": (i32, [vp, i32, vp, vp, vp]),
    "bamg_mlp_grad": (i32, [vp, i32, vp, vp, vp, vp, vp, vp]),
    "bamg_mlp_train": (i32, [vp, i32, vp, vp, vp, i32, i32, C.c_float, C.POINTER(C.c_float), vp]),
    "bamg_mlp_harvest": (i32, [vp, i32, vp, vp, vp, i32, ip, vp]),
    "bamg_vcycle_factor": (i32, [vp, i32, u64, dp, vp]),
    "bamg_setup_judged": (i32, [C.POINTER(Csr), C.POINTER(Params), f64, vp, C.POINTER(vp), dp, ip]),
    "bamg_num_levels": (i32, [vp]),
    "bamg_level": (i32, [vp, i32, C.POINTER(LevelView)]),
    "bamg_triplets": (i32, [vp, dp, ip, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
    "bamg_coarse_pinv": (i32, [vp, ip, C.POINTER(vp)]),
    "bamg_step_build_B_count": (i32, [i32, vp, vp, i64p, vp]),
    "bamg_step_build_B": (i32, [i32, vp, vp, vp, vp, vp, vp, vp]),
    "bamg_step_check_stochastic": (i32, [i32, vp, vp, vp, f64, i64p, vp]),
    "bamg_step_transpose": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
    "bamg_step_relax_block": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, f64, i32, vp]),
    "bamg_step_spmm_block": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp]),
    "bamg_step_jacobi_divisor": (i32, [i32, vp, vp, vp, vp, vp, vp, ip, vp]),
    "bamg_step_csr_vec": (i32, [i32, i32, i32, C.c_int64, vp, vp, vp, vp, f64, vp, vp, vp, vp]),
    "bamg_step_norms_weights": (i32, [i32, i32, i32, i32, vp, vp, vp, vp, i32, i32, dp, dp, vp]),
    "bamg_step_norms_weights_noalloc": (i32, [i32, i32, i32, i32, vp, vp, vp, vp, i32, i32, dp, dp, vp]),
    "bamg_step_coarsen_geometric": (i32, [i32, i32, vp, vp, vp, vp, ip, vp]),
    "bamg_step_coarsen_mis": (i32, [i32, vp, vp, vp, vp, u64, i32, vp, vp, ip, vp]),
    "bamg_step_graph_sets": (i32, [i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp]),
    "bamg_step_colour": (i32, [i32, vp, vp, vp, vp, u64, i32, vp, ip, vp]),
    "bamg_step_colour_rows": (i32, [i32, vp, i32, vp, vp, vp]),
    "bamg_step_mcgs_sweep": (i32, [i32, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]),
    "bamg_step_ls_fit": (i32, [i32, i32, i32, i32, vp, vp, vp, vp, i32, f64, vp, ip, vp]),
    "bamg_step_spgemm_symbolic": (i32, [i32, vp, vp, vp, vp, vp, i64p, vp]),
    "bamg_step_spgemm_numeric": (i32, [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "bamg_step_coarsest": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
}

_LIB = None


class BamgError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")
        self.status = status


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbamg is not built ({LIB_PATH} missing): run "
                               "`python -m paper_1402_4005_gb300.build` or __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status: int, where: str, allow=(0,)) -> int:
    if status not in allow:
        detail = lib().bamg_last_error().decode(errors="replace")
        raise BamgError(status, where, detail)
    return status
