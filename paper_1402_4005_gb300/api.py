"""Python binding of libbamg: the C ABI's calls under the same names.

Only argument marshalling happens here: device memory comes from PyTorch
tensors, every step of the method runs in the library's CUDA kernels.
Functions take and return ``torch`` tensors on the current CUDA device and
run on ``torch.cuda.current_stream()`` unless a stream is given.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

PREC = {"fp64": 0, "mixed": 1}


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _p(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


def _dev(x, dtype) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def bamg_params_default(**overrides) -> _lib.Params:
    p = _lib.Params()
    check(lib().bamg_params_default(C.byref(p)), "bamg_params_default")
    names = {"coarsening": {"geometric": 0, "mis": 1},
             "precision": {"fp64": 0, "mixed": 1},
             "restriction": {"ls": 0, "average": 1},
             "interp": {"ls": 0, "mlp": 1},
             "smoother": {"jacobi": 0, "mcgs": 1}}
    for k, v in overrides.items():
        if k in names and isinstance(v, str):
            v = names[k][v]
        if k == "mlp_params" and isinstance(v, torch.Tensor):
            # the caller keeps the tensor alive until bamg_setup returns
            if v.dtype != torch.float32 or not v.is_cuda or v.numel() != bamg_mlp_num_params():
                raise ValueError("mlp_params must be a CUDA float32 tensor of bamg_mlp_num_params() entries")
            v = v.data_ptr()
        setattr(p, k, v)
    return p


def bamg_solve_params_default(**overrides) -> _lib.SolveParams:
    p = _lib.SolveParams()
    check(lib().bamg_solve_params_default(C.byref(p)), "bamg_solve_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def launch_count() -> int:
    return int(lib().bamg_launch_count())


class Hierarchy:
    """A bamg_hierarchy handle; destroyed with the object when owned."""

    def __init__(self, handle: int, n: int, keep=(), owned: bool = True):
        self.handle = handle
        self.n = n
        self._keep = keep
        self._owned = owned

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "handle", None):
            if self._owned:
                lib().bamg_destroy(C.c_void_p(self.handle))
            self.handle = None

    def vcycle(self, r: torch.Tensor, stream=None) -> torch.Tensor:
        return bamg_vcycle(self, r, stream=stream)

    def solve(self, stream=None, **kw):
        return bamg_solve(self, stream=stream, **kw)

    @property
    def num_levels(self) -> int:
        return int(lib().bamg_num_levels(C.c_void_p(self.handle)))

    def level(self, l: int) -> dict:
        """Copies of the level's arrays (torch tensors on the device)."""
        v = _lib.LevelView()
        check(lib().bamg_level(C.c_void_p(self.handle), l, C.byref(v)), "bamg_level")
        torch.cuda.synchronize()
        out = {"n": v.n, "jacobi_l1_rows": v.jacobi_l1_rows}
        for name in ("B", "M", "N", "P", "Qt", "Q"):
            cv = getattr(v, name)
            out[name] = None if cv.rows == 0 else _csr_from_view(cv)
        if v.cf:
            out["cf"] = _copy_dev(v.cf, v.n, torch.int8)
            out["cmap"] = _copy_dev(v.cmap, v.n, torch.int32)
        if v.colour:
            out["colour"] = _copy_dev(v.colour, v.n, torch.int32)
            out["ncolours"] = v.ncolours
        return out

    def triplets(self, r: int) -> dict:
        sig = (C.c_double * r)()
        ld = C.c_int()
        U = C.c_void_p(); V = C.c_void_p(); x0 = C.c_void_p()
        check(lib().bamg_triplets(C.c_void_p(self.handle), sig, C.byref(ld), C.byref(U), C.byref(V),
                                  C.byref(x0)), "bamg_triplets")
        torch.cuda.synchronize()
        n, L = self.n, ld.value
        return {"sigma": np.array(sig[:]), "ld": L,
                "U": _copy_dev(U.value, n * L, torch.float64).view(n, L),
                "V": _copy_dev(V.value, n * L, torch.float64).view(n, L),
                "x0": _copy_dev(x0.value, n, torch.float64)}

    def coarse_pinv(self) -> torch.Tensor:
        nL = C.c_int(); ptr = C.c_void_p()
        check(lib().bamg_coarse_pinv(C.c_void_p(self.handle), C.byref(nL), C.byref(ptr)), "bamg_coarse_pinv")
        torch.cuda.synchronize()
        return _copy_dev(ptr.value, nL.value * nL.value, torch.float64).view(nL.value, nL.value)


class _DeviceArray:
    """A read-only device buffer described by __cuda_array_interface__."""

    def __init__(self, ptr: int, count: int, dtype):
        typestr = {torch.int8: "|i1", torch.int32: "<i4", torch.float64: "<f8", torch.float32: "<f4"}[dtype]
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _copy_dev(ptr: int, count: int, dtype) -> torch.Tensor:
    """Copy `count` elements at a library-owned device address into a new tensor."""
    if not count:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, count, dtype), device="cuda").clone()


def _csr_from_view(cv) -> dict:
    return {"rows": cv.rows, "cols": cv.cols, "nnz": cv.nnz,
            "row_ptr": _copy_dev(cv.row_ptr, cv.rows + 1, torch.int32),
            "col": _copy_dev(cv.col, cv.nnz, torch.int32),
            "val": _copy_dev(cv.val, cv.nnz, torch.float64)}


def _csr_struct(row_ptr, col, val, n, nx=0, ny=0, on_device=True):
    A = _lib.Csr()
    A.n = n
    A.nnz = int(col.shape[0])
    if on_device:
        A.row_ptr, A.col_idx, A.val = row_ptr.data_ptr(), col.data_ptr(), val.data_ptr()
    else:
        A.row_ptr = row_ptr.ctypes.data
        A.col_idx = col.ctypes.data
        A.val = val.ctypes.data
    A.on_device = 1 if on_device else 0
    A.nx, A.ny = nx, ny
    return A


def bamg_setup(row_ptr, col, val, n: int, params: _lib.Params | None = None, nx: int = 0, ny: int = 0,
               stream=None) -> Hierarchy:
    """Setup from a CSR of the column-stochastic A.

    Tensors on the GPU are read in place; numpy arrays are passed as host
    buffers (the library copies them to the device inside the call).
    """
    p = params if params is not None else bamg_params_default()
    if isinstance(row_ptr, torch.Tensor):
        rp, ci, va = _dev(row_ptr, torch.int32), _dev(col, torch.int32), _dev(val, torch.float64)
        A = _csr_struct(rp, ci, va, n, nx, ny, on_device=True)
        keep = (rp, ci, va)
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        va = np.ascontiguousarray(val, dtype=np.float64)
        A = _csr_struct(rp, ci, va, n, nx, ny, on_device=False)
        keep = (rp, ci, va)
    h = C.c_void_p()
    check(lib().bamg_setup(C.byref(A), C.byref(p), _stream(stream), C.byref(h)), "bamg_setup")
    return Hierarchy(h.value, n, keep=())


def bamg_vcycle(h: Hierarchy, r: torch.Tensor, z: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    r = _dev(r, torch.float64)
    z = torch.empty_like(r) if z is None else z
    check(lib().bamg_vcycle(C.c_void_p(h.handle), _p(r), _p(z), _stream(stream)), "bamg_vcycle")
    return z


def bamg_solve(h: Hierarchy, x: torch.Tensor | None = None, restart: int = 20, max_iter: int = 500,
               tol: float = 1e-10, stream=None, allow_not_converged: bool = False, plain: bool = False):
    """Returns (x, info dict); x > 0 with unit 1-norm.  plain: GMRES(restart)
    without the V-cycle from the uniform vector (the paper's comparator)."""
    x = torch.empty(h.n, dtype=torch.float64, device="cuda") if x is None else x
    sp = bamg_solve_params_default(restart=restart, max_iter=max_iter, tol=tol, plain=int(plain))
    info = _lib.SolveInfo()
    allow = (0, 5) if allow_not_converged else (0,)
    check(lib().bamg_solve(C.c_void_p(h.handle), _p(x), C.byref(sp), C.byref(info), _stream(stream)),
          "bamg_solve", allow)
    return x, info.as_dict()


def bamg_solve_host(row_ptr, col, val, n: int, params=None, nx: int = 0, ny: int = 0, restart: int = 20,
                    max_iter: int = 500, tol: float = 1e-10, stream=None):
    """Setup + solve from host arrays, x returned as a numpy array."""
    p = params if params is not None else bamg_params_default()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    A = _csr_struct(rp, ci, va, n, nx, ny, on_device=False)
    sp = bamg_solve_params_default(restart=restart, max_iter=max_iter, tol=tol)
    x = np.empty(n, dtype=np.float64)
    info = _lib.SolveInfo()
    check(lib().bamg_solve_host(C.byref(A), C.byref(p), C.byref(sp),
                                x.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info), _stream(stream)),
          "bamg_solve_host")
    return x, info.as_dict()


# ------------------------------------------------------------------- batches
class Batch:
    """Owner of a bamg_batch handle: many chains, one batched V-cycle and GMRES."""

    def __init__(self, handle: int, nchains: int, offsets: np.ndarray, keep=()):
        self.handle = handle
        self.nchains = nchains
        self.offsets = offsets
        self.n = int(offsets[-1])
        self._keep = keep

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "handle", None):
            lib().bamg_destroy_batched(C.c_void_p(self.handle))
            self.handle = None

    def chain(self, c: int) -> Hierarchy:
        h = lib().bamg_batch_chain(C.c_void_p(self.handle), c)
        n = int(self.offsets[c + 1] - self.offsets[c])
        return Hierarchy(h, n, owned=False)

    def lanes(self, level: int):
        b, p, q = C.c_int(), C.c_int(), C.c_int()
        check(lib().bamg_batch_lanes(C.c_void_p(self.handle), level, C.byref(b), C.byref(p), C.byref(q)),
              "bamg_batch_lanes")
        return b.value, p.value, q.value


def bamg_setup_batched(chains, params=None, host_threads: int = 0, stream=None) -> Batch:
    """chains: sequence of (row_ptr, col, val, n, nx, ny) host arrays."""
    p = params if params is not None else bamg_params_default()
    arr = (_lib.Csr * len(chains))()
    keep = []
    for k, (rp, ci, va, n, nx, ny) in enumerate(chains):
        rp = np.ascontiguousarray(rp, dtype=np.int32)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        va = np.ascontiguousarray(va, dtype=np.float64)
        keep += [rp, ci, va]
        arr[k] = _csr_struct(rp, ci, va, n, nx, ny, on_device=False)
    h = C.c_void_p()
    check(lib().bamg_setup_batched(arr, len(chains), C.byref(p), host_threads, _stream(stream), C.byref(h)),
          "bamg_setup_batched")
    off = np.zeros(len(chains) + 1, dtype=np.int64)
    check(lib().bamg_batch_offsets(h, off.ctypes.data_as(C.POINTER(C.c_int64))), "bamg_batch_offsets")
    return Batch(h.value, len(chains), off)


def bamg_solve_batched(b: Batch, restart: int = 20, max_iter: int = 500, tol: float = 1e-10, stream=None):
    """Returns (x concatenated in input order, list of per-chain info dicts)."""
    x = torch.empty(b.n, dtype=torch.float64, device="cuda")
    sp = bamg_solve_params_default(restart=restart, max_iter=max_iter, tol=tol)
    infos = (_lib.SolveInfo * b.nchains)()
    check(lib().bamg_solve_batched(C.c_void_p(b.handle), _p(x), C.byref(sp), C.cast(infos, C.c_void_p),
                                   _stream(stream)), "bamg_solve_batched")
    return x, [infos[k].as_dict() for k in range(b.nchains)]


def bamg_vcycle_batched(b: Batch, r: torch.Tensor, stream=None) -> torch.Tensor:
    r = _dev(r, torch.float64)
    z = torch.empty_like(r)
    check(lib().bamg_vcycle_batched(C.c_void_p(b.handle), _p(r), _p(z), _stream(stream)), "bamg_vcycle_batched")
    return z


# --------------------------------------------------------------------- steps
def bamg_step_build_B(A_rp: torch.Tensor, A_ci: torch.Tensor, A_val: torch.Tensor, stream=None):
    n = A_rp.shape[0] - 1
    nnz = C.c_int64()
    check(lib().bamg_step_build_B_count(n, _p(A_rp), _p(A_ci), C.byref(nnz), _stream(stream)), "build_B_count")
    rp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(nnz.value, dtype=torch.int32, device="cuda")
    va = torch.empty(nnz.value, dtype=torch.float64, device="cuda")
    check(lib().bamg_step_build_B(n, _p(A_rp), _p(A_ci), _p(A_val), _p(rp), _p(ci), _p(va), _stream(stream)),
          "build_B")
    return rp, ci, va


def bamg_step_check_stochastic(A_rp, A_ci, A_val, tol=1e-12, stream=None) -> int:
    bad = C.c_int64()
    check(lib().bamg_step_check_stochastic(A_rp.shape[0] - 1, _p(A_rp), _p(A_ci), _p(A_val), tol, C.byref(bad),
                                           _stream(stream)), "check_stochastic")
    return bad.value


def bamg_step_transpose(rp, ci, val, rows: int, cols: int, stream=None):
    nnz = ci.shape[0]
    trp = torch.empty(cols + 1, dtype=torch.int32, device="cuda")
    tci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    tva = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    check(lib().bamg_step_transpose(rows, cols, nnz, _p(rp), _p(ci), _p(val), _p(trp), _p(tci), _p(tva),
                                    _stream(stream)), "transpose")
    return trp, tci[:nnz], tva[:nnz]


def bamg_step_relax_block(rp, ci, val, dinv, X, R=None, sigma=None, omega=0.7, keep_col0=False, stream=None):
    prec = 1 if X.dtype == torch.float32 else 0
    n, ld = X.shape
    Y = torch.empty_like(X)
    check(lib().bamg_step_relax_block(prec, n, ld, _p(rp), _p(ci), _p(val), _p(dinv), _p(X), _p(Y), _p(R),
                                      _p(sigma), omega, int(keep_col0), _stream(stream)), "relax_block")
    return Y


def bamg_step_jacobi_divisor(rp, ci, val, trp, tval, stream=None):
    """(dinv, number of rows that took the l1 divisor) of a square CSR B."""
    n = rp.shape[0] - 1
    dinv = torch.empty(n, dtype=torch.float64, device="cuda")
    ns = C.c_int(0)
    check(lib().bamg_step_jacobi_divisor(n, _p(rp), _p(ci), _p(val), _p(trp), _p(tval), _p(dinv), C.byref(ns),
                                         _stream(stream)), "jacobi_divisor")
    return dinv, ns.value


def bamg_step_spmm_block(rp, ci, val, X, rows: int, stream=None):
    prec = 1 if X.dtype == torch.float32 else 0
    ld = X.shape[1]
    Y = torch.empty((rows, ld), dtype=X.dtype, device="cuda")
    check(lib().bamg_step_spmm_block(prec, rows, ld, _p(rp), _p(ci), _p(val), _p(X), _p(Y), _stream(stream)),
          "spmm_block")
    return Y


VEC_MODES = {"jacobi": 0, "jacobi_zero": 1, "resid": 2, "spmv": 3, "spmv_add": 4, "jacobi_zero2": 5}


def bamg_step_csr_vec(mode: str, rp, ci, val, x=None, b=None, dinv=None, omega=0.7, y=None, stream=None):
    """One launch of the V-cycle / GMRES vector kernel (see bamg_steps.h)."""
    ref = x if x is not None else b
    prec = 1 if ref.dtype == torch.float32 else 0
    n = rp.shape[0] - 1
    if y is None:
        y = torch.zeros(n, dtype=ref.dtype, device="cuda")
    check(lib().bamg_step_csr_vec(prec, VEC_MODES[mode], n, int(ci.shape[0]), _p(rp), _p(ci), _p(val), _p(dinv),
                                  float(omega), _p(x), _p(b), _p(y), _stream(stream)), "csr_vec")
    return y


def bamg_step_norms_weights(rp, ci, val, X, r: int, normalise=True, skip_col0=False, stream=None):
    prec = 1 if X.dtype == torch.float32 else 0
    n, ld = X.shape
    nrm = (C.c_double * r)()
    w = (C.c_double * r)()
    check(lib().bamg_step_norms_weights(prec, n, ld, r, _p(rp), _p(ci), _p(val), _p(X), int(normalise),
                                        int(skip_col0), nrm, w, _stream(stream)), "norms_weights")
    return np.array(nrm[:]), np.array(w[:])


def bamg_step_norms_weights_noalloc(rp, ci, val, X, r: int, normalise=True, skip_col0=False, stream=None):
    """bamg_step_norms_weights with fixed scratch (no device allocation inside)."""
    prec = 1 if X.dtype == torch.float32 else 0
    n, ld = X.shape
    nrm = (C.c_double * r)()
    w = (C.c_double * r)()
    check(lib().bamg_step_norms_weights_noalloc(prec, n, ld, r, _p(rp), _p(ci), _p(val), _p(X), int(normalise),
                                                int(skip_col0), nrm, w, _stream(stream)), "norms_weights_noalloc")
    return np.array(nrm[:]), np.array(w[:])


def bamg_step_coarsen_geometric(nx: int, ny: int, stream=None):
    n = nx * ny
    cf = torch.empty(n, dtype=torch.int8, device="cuda")
    cmap = torch.empty(n, dtype=torch.int32, device="cuda")
    jrp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    jci = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    nc = C.c_int()
    check(lib().bamg_step_coarsen_geometric(nx, ny, _p(cf), _p(cmap), _p(jrp), _p(jci), C.byref(nc),
                                            _stream(stream)), "coarsen_geometric")
    torch.cuda.current_stream().synchronize()
    return cf, cmap, jrp, jci[:int(jrp[-1].item())], nc.value


def bamg_step_coarsen_mis(B_rp, B_ci, Bt_rp, Bt_ci, seed: int, level: int, stream=None):
    n = B_rp.shape[0] - 1
    cf = torch.empty(n, dtype=torch.int8, device="cuda")
    cmap = torch.empty(n, dtype=torch.int32, device="cuda")
    nc = C.c_int()
    check(lib().bamg_step_coarsen_mis(n, _p(B_rp), _p(B_ci), _p(Bt_rp), _p(Bt_ci), seed, level, _p(cf), _p(cmap),
                                      C.byref(nc), _stream(stream)), "coarsen_mis")
    return cf, cmap, nc.value


def bamg_step_colour(B_rp, B_ci, Bt_rp, Bt_ci, seed: int, level: int, stream=None):
    """(colour[n] int32 device tensor, number of colours) of the symmetrised graph."""
    n = B_rp.shape[0] - 1
    colour = torch.empty(n, dtype=torch.int32, device="cuda")
    nc = C.c_int()
    check(lib().bamg_step_colour(n, _p(B_rp), _p(B_ci), _p(Bt_rp), _p(Bt_ci), seed, level, _p(colour), C.byref(nc),
                                 _stream(stream)), "colour")
    return colour, nc.value


def bamg_step_colour_rows(colour, ncolours: int, stream=None):
    """(colour offsets as a host numpy int32 array of ncolours + 1, rows tensor)."""
    import numpy as np
    n = colour.shape[0]
    crp = np.zeros(ncolours + 1, dtype=np.int32)
    rows = torch.empty(n, dtype=torch.int32, device="cuda")
    check(lib().bamg_step_colour_rows(n, _p(colour), ncolours, crp.ctypes.data, _p(rows), _stream(stream)),
          "colour_rows")
    return crp, rows


def bamg_step_mcgs_sweep(rp, ci, val, dinv, crp, rows, b, x, stream=None):
    """One multicolour Gauss-Seidel sweep on x in place (float32 or float64)."""
    import numpy as np
    prec = 1 if x.dtype == torch.float32 else 0
    crp = np.ascontiguousarray(crp, dtype=np.int32)
    check(lib().bamg_step_mcgs_sweep(prec, x.shape[0], _p(rp), _p(ci), _p(val), _p(dinv), crp.shape[0] - 1,
                                     crp.ctypes.data, _p(rows), _p(b), _p(x), _stream(stream)), "mcgs_sweep")
    return x


def bamg_step_graph_sets(B_rp, B_ci, B_val, Bt_rp, Bt_ci, Bt_val, cf, c_min: int, c_max: int, stream=None):
    n = B_rp.shape[0] - 1
    jrp = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    jci = torch.empty(max(n * c_max, 1), dtype=torch.int32, device="cuda")
    check(lib().bamg_step_graph_sets(n, _p(B_rp), _p(B_ci), _p(B_val), _p(Bt_rp), _p(Bt_ci), _p(Bt_val), _p(cf),
                                     c_min, c_max, _p(jrp), _p(jci), _stream(stream)), "graph_sets")
    torch.cuda.current_stream().synchronize()
    return jrp, jci[:int(jrp[-1].item())]


def bamg_step_ls_fit(J_rp, J_ci, X, w, r: int, constrained=False, ridge: float = 0.0, stream=None):
    prec = 1 if X.dtype == torch.float32 else 0
    n, ld = X.shape
    nnz = J_ci.shape[0]
    out = torch.zeros(max(nnz, 1), dtype=torch.float64, device="cuda")
    rk = C.c_int()
    w = _dev(w, torch.float64)
    check(lib().bamg_step_ls_fit(prec, n, ld, r, _p(J_rp), _p(J_ci), _p(X), _p(w), int(constrained),
                                 float(ridge), _p(out), C.byref(rk), _stream(stream)), "ls_fit")
    return out[:nnz], rk.value


def bamg_step_spgemm(A_rp, A_ci, A_val, B_rp, B_ci, B_val, stream=None):
    m = A_rp.shape[0] - 1
    crp = torch.empty(m + 1, dtype=torch.int32, device="cuda")
    nnz = C.c_int64()
    check(lib().bamg_step_spgemm_symbolic(m, _p(A_rp), _p(A_ci), _p(B_rp), _p(B_ci), _p(crp), C.byref(nnz),
                                          _stream(stream)), "spgemm_symbolic")
    cci = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
    cva = torch.empty(max(nnz.value, 1), dtype=torch.float64, device="cuda")
    check(lib().bamg_step_spgemm_numeric(m, _p(A_rp), _p(A_ci), _p(A_val), _p(B_rp), _p(B_ci), _p(B_val),
                                         _p(crp), _p(cci), _p(cva), _stream(stream)), "spgemm_numeric")
    return crp, cci[:nnz.value], cva[:nnz.value]


def bamg_step_coarsest(B, M, N, r: int, prec: str = "fp64", pinv=True, stream=None):
    n = B.shape[0]
    B, M, N = (_dev(t, torch.float64) for t in (B, M, N))
    sig = torch.empty(r, dtype=torch.float64, device="cuda")
    U = torch.empty((n, r), dtype=torch.float64, device="cuda")
    V = torch.empty((n, r), dtype=torch.float64, device="cuda")
    P = torch.empty((n, n), dtype=torch.float64, device="cuda") if pinv else None
    check(lib().bamg_step_coarsest(PREC[prec], n, r, _p(B), _p(M), _p(N), _p(sig), _p(U), _p(V), _p(P),
                                   _stream(stream)), "coarsest")
    return sig, U, V, P


# ------------------------------------------------------ learned interpolation
def bamg_mlp_num_params() -> int:
    return int(lib().bamg_mlp_num_params())


def bamg_mlp_init(seed: int = 5, stream=None) -> torch.Tensor:
    """Fresh network parameters (float32 vector on the GPU)."""
    p = torch.empty(bamg_mlp_num_params(), dtype=torch.float32, device="cuda")
    check(lib().bamg_mlp_init(_p(p), C.c_uint64(seed), _stream(stream)), "bamg_mlp_init")
    return p


def bamg_mlp_save(params: torch.Tensor, path: str, stream=None) -> None:
    """Write a parameter vector (CUDA or CPU float32 tensor) to a file."""
    if params.dtype != torch.float32 or params.numel() != bamg_mlp_num_params() or not params.is_contiguous():
        raise ValueError("params must be a contiguous float32 tensor of bamg_mlp_num_params() entries")
    dev = 1 if params.is_cuda else 0
    check(lib().bamg_mlp_save(str(path).encode(), _p(params), dev, _stream(stream) if dev else None),
          "bamg_mlp_save")


def bamg_mlp_load(path: str, device: str = "cuda", stream=None) -> torch.Tensor:
    """Parameter vector read from a file, on the GPU (default) or the CPU."""
    p = torch.empty(bamg_mlp_num_params(), dtype=torch.float32, device=device)
    dev = 1 if p.is_cuda else 0
    check(lib().bamg_mlp_load(str(path).encode(), _p(p), dev, _stream(stream) if dev else None),
          "bamg_mlp_load")
    return p


def _bf16_rows(X) -> torch.Tensor:
    X = X if isinstance(X, torch.Tensor) else torch.as_tensor(np.asarray(X, dtype=np.float32))
    X = X.to(device="cuda", dtype=torch.bfloat16).contiguous()
    if X.dim() != 2 or X.shape[1] != 64:
        raise ValueError("features must be an M x 64 array")
    return X


def bamg_mlp_forward(params: torch.Tensor, X, stream=None) -> torch.Tensor:
    X = _bf16_rows(X)
    Y = torch.empty(X.shape[0], 16, dtype=torch.float32, device="cuda")
    check(lib().bamg_mlp_forward(_p(params), X.shape[0], _p(X), _p(Y), _stream(stream)), "bamg_mlp_forward")
    return Y


def bamg_mlp_grad(params: torch.Tensor, X, T, mask, stream=None):
    """(loss, gradient) of the masked mean squared error."""
    X = _bf16_rows(X)
    T = _dev(T, torch.float32)
    mask = _dev(mask, torch.float32)
    g = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    check(lib().bamg_mlp_grad(_p(params), X.shape[0], _p(X), _p(T), _p(mask), _p(g), _p(loss),
                              _stream(stream)), "bamg_mlp_grad")
    return float(loss.item()), g


def bamg_mlp_train(params: torch.Tensor, X, T, mask, epochs: int = 10, batch: int = 4096, lr: float = 1e-3,
                   stream=None) -> list:
    """Adam on the network in place; returns the mean loss of each epoch."""
    X = _bf16_rows(X)
    T = _dev(T, torch.float32)
    mask = _dev(mask, torch.float32)
    losses = (C.c_float * epochs)()
    check(lib().bamg_mlp_train(_p(params), X.shape[0], _p(X), _p(T), _p(mask), epochs, batch, C.c_float(lr),
                               losses, _stream(stream)), "bamg_mlp_train")
    return list(losses)


def bamg_mlp_harvest(h: Hierarchy, level: int, stream=None):
    """(X bf16 [nF, 64], T [nF, 16], mask [nF, 16]) of a level of an LS hierarchy."""
    cnt = C.c_int(0)
    check(lib().bamg_mlp_harvest(C.c_void_p(h.handle), level, None, None, None, 0, C.byref(cnt),
                                 _stream(stream)), "bamg_mlp_harvest")
    nf = cnt.value
    X = torch.empty(max(nf, 1), 64, dtype=torch.bfloat16, device="cuda")
    T = torch.empty(max(nf, 1), 16, dtype=torch.float32, device="cuda")
    M = torch.empty(max(nf, 1), 16, dtype=torch.float32, device="cuda")
    check(lib().bamg_mlp_harvest(C.c_void_p(h.handle), level, _p(X), _p(T), _p(M), max(nf, 1), C.byref(cnt),
                                 _stream(stream)), "bamg_mlp_harvest")
    return X[:nf], T[:nf], M[:nf]


def bamg_vcycle_factor(h: Hierarchy, iters: int = 12, seed: int = 1, stream=None) -> float:
    f = C.c_double(0.0)
    check(lib().bamg_vcycle_factor(C.c_void_p(h.handle), iters, C.c_uint64(seed), C.byref(f), _stream(stream)),
          "bamg_vcycle_factor")
    return f.value


def bamg_setup_judged(row_ptr, col, val, n: int, params: _lib.Params, max_factor: float, nx: int = 0,
                      ny: int = 0, stream=None):
    """Learned setup with the LS fallback: (Hierarchy, factor, used_ls)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    A = _csr_struct(rp, ci, va, n, nx, ny, on_device=False)
    h = C.c_void_p()
    f = C.c_double(0.0)
    used = C.c_int(0)
    check(lib().bamg_setup_judged(C.byref(A), C.byref(params), C.c_double(max_factor), _stream(stream),
                                  C.byref(h), C.byref(f), C.byref(used)), "bamg_setup_judged")
    return Hierarchy(h.value, n), f.value, bool(used.value)
