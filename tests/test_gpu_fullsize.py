"""Parity of the block kernels at the sizes where the library switches to its
large-level layout (n >= 2^17 rows: two interleaved 16-byte vectors per lane),
and error behaviour of the least-squares step.

The relaxation and block SpMM are checked against the oracle's weighted
Jacobi sweep and sparse product on a 2^17 + 37-point Delaunay walk
(irregular rows, ragged tail) and a 400^2 tandem queue, in both
precisions and at every block width that takes the interleaved layout
(FP32: 16, 32; FP64: 8, 16, 32), with the componentwise-scaled error
|y - y*| / (|B||x| + |b|) at 1e-12 (FP64) and 1e-5 (FP32).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import chaingen as cg
from oracle import operators, rng, smoothing

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def scaled_err(y, ystar, B, x, b=None):
    den = abs(B) @ np.abs(x)
    if b is not None:
        den = den + np.abs(b)
    den = np.maximum(den, np.finfo(float).tiny)
    return np.max(np.abs(y - ystar) / den)


_CH = {}


def chain(name):
    if name not in _CH:
        ch = cg.delaunay_walk((1 << 17) + 37, seed=11) if name == "delaunay" else cg.tandem(400)
        B = operators.build_B(ch.csr())
        B.sort_indices()
        _CH[name] = (ch, B, operators.diag(B))
    return _CH[name]


CASES = [("fp32", 16), ("fp32", 32), ("fp64", 8), ("fp64", 16), ("fp64", 32)]


@pytest.mark.parametrize("name", ["delaunay", "tandem"])
@pytest.mark.parametrize("prec,ld", CASES)
def test_relax_block_large_levels(api, name, prec, ld):
    ch, B, d = chain(name)
    n = ch.n
    assert n >= 1 << 17
    r = ld - 3
    X = np.zeros((n, ld)); R = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(21, 2 * k, n)
        R[:, k] = rng.uniform_pm1(21, 2 * k + 1, n)
    sig = np.zeros(ld); sig[:r] = np.linspace(0.05, 1.5, r)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    rp, ci = dev(B.indptr.astype(np.int32)), dev(B.indices.astype(np.int32))
    va = dev(B.data).to(dt)
    dinv = dev(1.0 / d).to(dt)
    Xd = dev(X).to(dt)
    Y = api.bamg_step_relax_block(rp, ci, va, dinv, Xd, keep_col0=True).double().cpu().numpy()
    Ys = smoothing.jacobi(B, d, X, None, 0.7)
    Ys[:, 0] = X[:, 0]
    assert scaled_err(Y, Ys, B, X) <= tol
    assert np.all(Y[:, r:] == 0.0)                      # padding columns stay zero
    Rs = R * sig[None, :]
    Y = api.bamg_step_relax_block(rp, ci, va, dinv, Xd, R=dev(R).to(dt),
                                  sigma=dev(sig).to(dt)).double().cpu().numpy()
    Ys = smoothing.jacobi(B, d, X, Rs, 0.7)
    assert scaled_err(Y, Ys, B, X, Rs) <= tol
    # a prefix of the rows (the product of a level's leading rows)
    Y = api.bamg_step_spmm_block(rp, ci, va, Xd, n).double().cpu().numpy()
    assert scaled_err(Y, B @ X, B, X) <= tol


def test_ls_fit_rejects_oversized_sets(api):
    """Sets larger than min(ld, 8) cannot be fitted: BAMG_ERR_ARG, and the
    rows with admissible sets are still fitted."""
    from paper_1402_4005_gb300._lib import BamgError
    n, ld, r = 64, 4, 4
    X = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(5, k, n)
    rp = [0]; ci = []
    for i in range(n):
        c = 5 if i == 10 else (2 if i % 2 else 0)
        ci.extend(range(20, 20 + c)); rp.append(len(ci))
    w = np.ones(ld)
    with pytest.raises(BamgError):
        api.bamg_step_ls_fit(dev(np.array(rp, np.int32)), dev(np.array(ci, np.int32)), dev(X), w, r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ls_fit_counts_rank_deficient_rows_once(api, prec):
    """A set that names the same coarse point twice gives two equal columns:
    the fit is rank deficient.  In FP32 such a row fails the condition test,
    is refitted in FP64 and must still be counted once."""
    n, ld, r = 300, 8, 8
    X = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(6, k, n)
    rp = [0]; ci = []
    dup = 0
    for i in range(n):
        if i % 3 == 0:
            cols = [(i + 1) % n, (i + 1) % n, (i + 5) % n]
            dup += 1
        elif i % 3 == 1:
            cols = [(i + 2) % n, (i + 7) % n]
        else:
            cols = []
        ci.extend(cols); rp.append(len(ci))
    dt = torch.float64 if prec == "fp64" else torch.float32
    fit, rk = api.bamg_step_ls_fit(dev(np.array(rp, np.int32)), dev(np.array(ci, np.int32)),
                                   dev(X).to(dt), np.ones(ld), r)
    assert rk == dup
    fit = fit.cpu().numpy()
    # the full-rank rows match the plain least-squares solution
    for i in range(1, n, 3):
        a, b = rp[i], rp[i + 1]
        A = X[ci[a:b], :r].T
        ref = np.linalg.lstsq(A, X[i, :r], rcond=None)[0]
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert np.abs(fit[a:b] - ref).max() <= tol * np.linalg.cond(A) * 10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("name", ["small", "delaunay", "tandem"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_csr_vec_modes_against_oracle(api, name, prec):
    """The V-cycle / GMRES vector kernel in all six modes against the
    oracle's Jacobi sweeps and sparse products (1e-12 / 1e-5 scaled); the
    two sweeps from zero in one pass bit for bit equal to the two launches."""
    if name == "small":
        ch = cg.delaunay_walk(2999, seed=12)
        B = operators.build_B(ch.csr()); B.sort_indices()
        d = operators.diag(B)
    else:
        ch, B, d = chain(name)
    n = ch.n
    x = rng.uniform_pm1(31, 0, n)
    b = rng.uniform_pm1(31, 1, n)
    y0 = rng.uniform_pm1(31, 2, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    rp, ci = dev(B.indptr.astype(np.int32)), dev(B.indices.astype(np.int32))
    va = dev(B.data).to(dt)
    xd, bd, dinv = dev(x).to(dt), dev(b).to(dt), dev(1.0 / d).to(dt)
    got = lambda mode, **k: api.bamg_step_csr_vec(mode, rp, ci, va, **k).double().cpu().numpy()
    ref = smoothing.jacobi(B, d, x[:, None], b[:, None], 0.7)[:, 0]
    assert scaled_err(got("jacobi", x=xd, b=bd, dinv=dinv), ref, B, x, b) <= tol
    assert np.abs(got("jacobi_zero", b=bd, dinv=dinv) - 0.7 * b / d).max() <= tol * np.abs(b / d).max()
    assert scaled_err(got("resid", x=xd, b=bd), b - B @ x, B, x, b) <= tol
    assert scaled_err(got("spmv", x=xd), B @ x, B, x) <= tol
    y = dev(y0).to(dt)
    api.bamg_step_csr_vec("spmv_add", rp, ci, va, x=xd, y=y)
    assert scaled_err(y.double().cpu().numpy(), y0 + B @ x, B, x, y0) <= tol
    z1 = api.bamg_step_csr_vec("jacobi_zero", rp, ci, va, b=bd, dinv=dinv)
    z2 = api.bamg_step_csr_vec("jacobi", rp, ci, va, x=z1, b=bd, dinv=dinv)
    z2f = api.bamg_step_csr_vec("jacobi_zero2", rp, ci, va, b=bd, dinv=dinv)
    assert torch.equal(z2f, z2)
    r1 = smoothing.jacobi(B, d, np.zeros((n, 1)), b[:, None], 0.7)
    r2 = smoothing.jacobi(B, d, r1, b[:, None], 0.7)[:, 0]
    assert scaled_err(z2f.double().cpu().numpy(), r2, B, r1[:, 0], b) <= tol
