"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^\s*(?:bamg_status|void|const char\*|uint64_t|int|bamg_hierarchy\*)\s+(bamg_\w+)\s*\(",
                                src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function has a binding signature with the same name
    assert names == set(_lib.SIGNATURES), names ^ set(_lib.SIGNATURES)


def test_status_strings_without_gpu():
    from paper_1402_4005_gb300 import _lib
    L = _lib.lib()
    assert L.bamg_status_string(0) == b"ok"
    assert L.bamg_status_string(2) == b"matrix is not column stochastic"
    p = _lib.Params()
    assert L.bamg_params_default(ctypes.byref(p)) == 0
    assert (p.r, p.nu_pre, p.nu_post, round(p.omega, 12)) == (8, 3, 3, 0.7)
    assert L.bamg_setup(None, None, None, None) == 1      # BAMG_ERR_ARG, no device touched


def test_parameter_structs_match_the_header():
    """bamg_params_default zeroes the whole C struct before setting the
    defaults: bytes past the binding's struct must stay untouched (the two
    layouts agree), and the defaults of the later fields are as declared."""
    from paper_1402_4005_gb300 import _lib
    L = _lib.lib()
    size = ctypes.sizeof(_lib.Params)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    assert L.bamg_params_default(ctypes.cast(buf, ctypes.POINTER(_lib.Params))) == 0
    assert all(b == 0xAB for b in buf[size:]), "bamg_params is larger in the header than in the binding"
    p = _lib.Params.from_buffer(buf)
    assert (p.setup_cycles, p.interp, p.smoother, p.max_coarse_dense, p.ls_ridge) == (1, 0, 0, 1024, 0.0)
    assert p.mlp_params is None
    sp = _lib.SolveParams()
    sp.plain = 7
    assert L.bamg_solve_params_default(ctypes.byref(sp)) == 0
    assert (sp.restart, sp.max_iter, sp.tol, sp.plain) == (20, 500, 1e-10, 0)


def test_penalty_weight_is_validated_before_any_device_call():
    """bamg_params.ls_ridge must be finite and >= 0; the check runs before
    the library touches a device, so it needs no GPU."""
    import numpy as np
    from paper_1402_4005_gb300 import _lib
    L = _lib.lib()
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([1, 0], np.int32)
    va = np.array([1.0, 1.0])
    A = _lib.Csr(n=2, nnz=2, row_ptr=rp.ctypes.data, col_idx=ci.ctypes.data, val=va.ctypes.data,
                 on_device=0, nx=2, ny=1)
    for bad in (-0.5, float("nan"), float("inf")):
        p = _lib.Params()
        assert L.bamg_params_default(ctypes.byref(p)) == 0
        p.ls_ridge = bad
        out = ctypes.c_void_p()
        assert L.bamg_setup(ctypes.byref(A), ctypes.byref(p), None, ctypes.byref(out)) == 1, bad
        assert not out.value
