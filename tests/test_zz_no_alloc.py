"""The allocation-free norms/weights entry point against the regular one.

bamg_step_norms_weights_noalloc serves callers that may not allocate device
memory while running (their memory is planned up front); it keeps its
scratch in a fixed device array.  Two calls in a row must reproduce the
results of bamg_step_norms_weights within the tolerances of the other
kernel tests (1e-12 in FP64, 1e-5 in FP32), including the in-place
normalisation of the block.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import chaingen as cg
from oracle import operators, rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api as a
    return a


def _block(n, ld, r, seed):
    X = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(seed, 2 * k, n)
    return X


@pytest.mark.parametrize("prec,ld,r,skip0", [("fp64", 16, 16, False), ("fp64", 8, 7, True),
                                             ("fp32", 16, 13, True), ("fp32", 32, 32, False)])
def test_noalloc_matches_regular_entry_point(api, prec, ld, r, skip0):
    ch = cg.tandem(61)                                  # n = 3721, ragged against the row tiles
    B = operators.build_B(ch.csr())
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    rp = torch.from_numpy(B.indptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(B.indices.astype(np.int32)).cuda()
    va = torch.from_numpy(B.data).cuda().to(dt)
    for call, seed in enumerate((4, 9)):                # two calls in a row, different data
        X = _block(ch.n, ld, r, seed)
        Xa = torch.from_numpy(X).cuda().to(dt)
        Xb = Xa.clone()
        n1, w1 = api.bamg_step_norms_weights(rp, ci, va, Xa, r, normalise=True, skip_col0=skip0)
        n2, w2 = api.bamg_step_norms_weights_noalloc(rp, ci, va, Xb, r, normalise=True, skip_col0=skip0)
        torch.cuda.synchronize()
        assert np.allclose(n2, n1, rtol=tol, atol=0), call
        assert np.allclose(w2, w1, rtol=tol, atol=0), call
        assert (w2[0] == 0.0) == skip0
        diff = (Xb.double() - Xa.double()).abs().max().item()
        assert diff <= tol, (call, diff)


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    from paper_1402_4005_gb300._lib import BamgError
    ch = cg.tandem(9)
    B = operators.build_B(ch.csr())
    rp = torch.from_numpy(B.indptr.astype(np.int32)).cuda()
    ci = torch.from_numpy(B.indices.astype(np.int32)).cuda()
    va = torch.from_numpy(B.data).cuda()
    X = torch.zeros((ch.n, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(BamgError) as e:
        api.bamg_step_norms_weights_noalloc(rp, ci, va, X, 8)
    assert e.value.status == 1
