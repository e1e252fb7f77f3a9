"""Per-kernel parity of the CUDA library against the CPU oracle.

Both sides receive the same seeded inputs (chaingen generators, SplitMix64
vectors, or oracle outputs); integer work must match bit for bit and
floating point within the stated tolerances:
  FP64: 1e-12 in the componentwise-scaled error |y - y*| / (|B||x| + |b|)
  FP32: 1e-5 in the same measure
  least-squares weights: 1e-12 * cond(weighted system), or 1e-5 (FP32 input)
"""
import numpy as np
import pytest
import scipy.sparse as sp

import chaingen as cg
from oracle import coarsening, coarsest, interp, operators, rng, smoothing

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api as a
    assert torch.cuda.is_available()
    return a


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def csr_dev(M: sp.csr_matrix, dtype=torch.float64):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return (dev(M.indptr.astype(np.int32)), dev(M.indices.astype(np.int32)),
            dev(M.data.astype(np.float64)).to(dtype))


def scaled_err(y, ystar, B, x, b=None):
    den = abs(B) @ np.abs(x)
    if b is not None:
        den = den + np.abs(b)
    den = np.maximum(den, np.finfo(float).tiny)
    return np.max(np.abs(y - ystar) / den)


CHAINS = {
    "lattice": lambda: cg.lattice2d(37, 29, seed=4),
    "tandem": lambda: cg.tandem(41),
    "delaunay": lambda: cg.delaunay_walk(3001, seed=5),
}


# ------------------------------------------------------------------ A1
@pytest.mark.parametrize("name", list(CHAINS))
def test_build_B_and_transpose_bit_exact(api, name):
    ch = CHAINS[name]()
    rp, ci, va = api.bamg_step_build_B(dev(ch.row_ptr), dev(ch.col), dev(ch.val))
    B = operators.build_B(ch.csr())
    assert np.array_equal(rp.cpu().numpy(), B.indptr)
    assert np.array_equal(ci.cpu().numpy(), B.indices)
    assert np.array_equal(va.cpu().numpy(), B.data)
    trp, tci, tva = api.bamg_step_transpose(rp, ci, va, ch.n, ch.n)
    Bt = operators.transpose(B)
    assert np.array_equal(trp.cpu().numpy(), Bt.indptr)
    assert np.array_equal(tci.cpu().numpy(), Bt.indices)
    assert np.array_equal(tva.cpu().numpy(), Bt.data)


def test_check_stochastic_flags_bad_columns(api):
    ch = cg.tandem(9)
    assert api.bamg_step_check_stochastic(dev(ch.row_ptr), dev(ch.col), dev(ch.val)) == 0
    bad = ch.val.copy()
    bad[5] *= 1.001
    bad[7] = -bad[7]
    assert api.bamg_step_check_stochastic(dev(ch.row_ptr), dev(ch.col), dev(bad)) >= 2


# ------------------------------------------------------------------ A6, A7
@pytest.mark.parametrize("ld", [4, 8, 16, 32])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_relax_block(api, ld, prec):
    ch = cg.delaunay_walk(2999, seed=7)     # irregular rows, ragged tail
    B = operators.build_B(ch.csr())
    d = operators.diag(B)
    n = ch.n
    r = ld - 1 if ld > 4 else ld
    X = np.zeros((n, ld)); R = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(3, 2 * k, n)
        R[:, k] = rng.uniform_pm1(3, 2 * k + 1, n)
    sig = np.zeros(ld); sig[:r] = np.linspace(0.1, 2.0, r)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    rp, ci, va = csr_dev(B, dt)
    dinv = dev(1.0 / d).to(dt)
    # homogeneous, keep column 0
    Y = api.bamg_step_relax_block(rp, ci, va, dinv, dev(X).to(dt), keep_col0=True).double().cpu().numpy()
    Ys = smoothing.jacobi(B, d, X, None, 0.7)
    Ys[:, 0] = X[:, 0]
    assert scaled_err(Y, Ys, B, X) <= tol
    # inhomogeneous: rhs sigma .* R
    Y = api.bamg_step_relax_block(rp, ci, va, dinv, dev(X).to(dt), R=dev(R).to(dt),
                                  sigma=dev(sig).to(dt)).double().cpu().numpy()
    Ys = smoothing.jacobi(B, d, X, R * sig[None, :], 0.7)
    assert scaled_err(Y, Ys, B, X, R * sig[None, :]) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spmm_and_norms_weights(api, prec):
    ch = cg.tandem(33)
    B = operators.build_B(ch.csr())
    n, ld, r = ch.n, 16, 13
    X = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(9, 2 * k, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    rp, ci, va = csr_dev(B, dt)
    Y = api.bamg_step_spmm_block(rp, ci, va, dev(X).to(dt), n).double().cpu().numpy()
    assert scaled_err(Y, B @ X, B, X) <= tol
    Xd = dev(X).to(dt)
    nrm, w = api.bamg_step_norms_weights(rp, ci, va, Xd, r, normalise=True, skip_col0=True)
    Xn = interp.normalise(X[:, :r], range(1, r))
    ws = interp.weights(B, Xn, range(1, r))
    assert np.allclose(nrm, np.linalg.norm(X[:, :r], axis=0), rtol=tol)
    assert w[0] == 0.0 and np.allclose(w[1:], ws[1:], rtol=10 * tol)
    assert np.allclose(Xd.double().cpu().numpy()[:, :r], Xn, rtol=0, atol=tol)


# ------------------------------------------------------------------ A2, A4
@pytest.mark.parametrize("nx,ny", [(16, 16), (17, 9), (2, 7), (33, 1)])
def test_geometric_coarsening_bit_exact(api, nx, ny):
    cf, cmap, jrp, jci, nc = api.bamg_step_coarsen_geometric(nx, ny)
    cfo, cmo, _ = coarsening.geometric(nx, ny)
    J = coarsening.geometric_sets(nx, ny, cfo)
    assert nc == int(cfo.sum())
    assert np.array_equal(cf.cpu().numpy().astype(bool), cfo)
    assert np.array_equal(cmap.cpu().numpy(), cmo)
    jrp, jci = jrp.cpu().numpy(), jci.cpu().numpy()
    for i in range(nx * ny):
        assert list(jci[jrp[i]:jrp[i + 1]]) == (J.get(i, []) if not cfo[i] else [])


def _graph(name):
    ch = CHAINS[name]()
    B = operators.build_B(ch.csr())
    return B, operators.transpose(B)


@pytest.mark.parametrize("name", ["delaunay", "tandem"])
def test_mis_bit_exact(api, name):
    B, Bt = _graph(name)
    for level, seed in ((0, 3), (2, 11)):
        cf, cmap, nc = api.bamg_step_coarsen_mis(*csr_dev(B)[:2], *csr_dev(Bt)[:2], seed, level)
        cfo, cmo = coarsening.greedy_mis(B, Bt, seed, level)
        assert np.array_equal(cf.cpu().numpy().astype(bool), cfo)
        assert np.array_equal(cmap.cpu().numpy(), cmo) and nc == int(cfo.sum())


@pytest.mark.parametrize("cmin,cmax", [(1, 4), (3, 8), (2, 2)])
def test_graph_sets_bit_exact(api, cmin, cmax):
    B, Bt = _graph("delaunay")
    cfo, _ = coarsening.greedy_mis(B, Bt, 1, 0)
    J = coarsening.graph_sets(B, Bt, cfo, cmin, cmax)
    jrp, jci = api.bamg_step_graph_sets(*csr_dev(B), *csr_dev(Bt), dev(cfo.astype(np.int8)), cmin, cmax)
    jrp, jci = jrp.cpu().numpy(), jci.cpu().numpy()
    for i in range(B.shape[0]):
        got = list(jci[jrp[i]:jrp[i + 1]])
        assert got == (J[i] if not cfo[i] else []), i


# ------------------------------------------------------------------ A8, A9
def _smoothed_vectors(B, d, n, r, ld, seed, sweeps=5, first_ones=False):
    X = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(seed, 2 * k, n)
    if first_ones:
        X[:, 0] = 1.0
    for _ in range(sweeps):
        Y = smoothing.jacobi(B, d, X, None, 0.7)
        if first_ones:
            Y[:, 0] = 1.0
        X = Y
    return X


def _J_csr(J, cf, n):
    rp = [0]; ci = []
    for i in range(n):
        if not cf[i]:
            ci.extend(J[i])
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32)


@pytest.mark.parametrize("geom,ld,r", [(True, 8, 8), (True, 16, 12), (False, 8, 8), (False, 16, 16)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ls_fits_against_oracle(api, geom, ld, r, prec):
    if geom:
        ch = cg.tandem(31)
        B = operators.build_B(ch.csr())
        cf, cmap, _ = coarsening.geometric(31, 31)
        J = coarsening.geometric_sets(31, 31, cf)
    else:
        ch = cg.delaunay_walk(2500, seed=8)
        B = operators.build_B(ch.csr())
        Bt = operators.transpose(B)
        cf, cmap = coarsening.greedy_mis(B, Bt, 2, 0)
        J = coarsening.graph_sets(B, Bt, cf, 3, 8 if ld >= 8 else 4)
    d = operators.diag(B)
    n = ch.n
    Bt = operators.transpose(B)
    V = interp.normalise(_smoothed_vectors(B, d, n, r, ld, 5)[:, :r])
    U = interp.normalise(_smoothed_vectors(Bt, d, n, r, ld, 6, first_ones=True)[:, :r], range(1, r))
    s = interp.weights(B, V)
    t = interp.weights(Bt, U, range(1, r))
    P = interp.ls_interpolation(V, s, cf, cmap, J)
    Qt = interp.ls_restriction_T(U, t, cf, cmap, J)
    jrp, jci = _J_csr(J, cf, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Vp = np.zeros((n, ld)); Vp[:, :r] = V
    Up = np.zeros((n, ld)); Up[:, :r] = U
    sp_ = np.zeros(ld); sp_[:r] = s
    tp_ = np.zeros(ld); tp_[:r] = t
    fitP, rk1 = api.bamg_step_ls_fit(dev(jrp), dev(jci), dev(Vp).to(dt), sp_, r)
    fitQ, rk2 = api.bamg_step_ls_fit(dev(jrp), dev(jci), dev(Up).to(dt), tp_, r, constrained=True)
    fitP, fitQ = fitP.cpu().numpy(), fitQ.cpu().numpy()
    assert rk1 == 0 and rk2 == 0
    for i in range(n):
        if cf[i]:
            continue
        a, b = jrp[i], jrp[i + 1]
        cols = cmap[J[i]]
        Xw = V[J[i], :].T * s[:, None]
        kap = np.linalg.cond(Xw) if Xw.shape[1] > 1 else 1.0
        tol = (1e-12 * kap * 10 if prec == "fp64" else 1e-5 * kap * 10)
        pr = P[i, cols].toarray().ravel()
        assert np.abs(fitP[a:b] - pr).max() <= tol * max(1.0, np.abs(pr).max()), (i, kap)
        qr = Qt[i, cols].toarray().ravel()
        Uw = U[J[i], 1:].T * t[1:, None]
        kq = np.linalg.cond(Uw) if Uw.shape[1] > 1 else 1.0
        tq = (1e-12 * kq * 10 if prec == "fp64" else 1e-5 * kq * 10)
        assert np.abs(fitQ[a:b] - qr).max() <= tq * max(1.0, np.abs(qr).max()), (i, kq)
        assert abs(fitQ[a:b].sum() - 1.0) <= 1e-13 * len(J[i])


# ------------------------------------------------------------------ A10
@pytest.mark.parametrize("case", ["galerkin", "random"])
def test_spgemm_pattern_exact_values_close(api, case):
    if case == "random":
        X = sp.random(700, 500, density=0.01, random_state=3, format="csr")
        Y = sp.random(500, 650, density=0.012, random_state=4, format="csr")
        pairs = [(X, Y)]
    else:
        ch = cg.lattice2d(23, 19, seed=2)
        B = operators.build_B(ch.csr())
        cf, cmap, _ = coarsening.geometric(23, 19)
        J = coarsening.geometric_sets(23, 19, cf)
        n = ch.n
        V = interp.normalise(_smoothed_vectors(B, operators.diag(B), n, 8, 8, 3)[:, :8])
        P = interp.ls_interpolation(V, interp.weights(B, V), cf, cmap, J)
        Q = operators.transpose(P)
        pairs = [(B, P), (Q, operators.spmatmul(B, P)), (Q, P.copy())]
    for X, Y in pairs:
        X = sp.csr_matrix(X); X.sort_indices()
        Y = sp.csr_matrix(Y); Y.sort_indices()
        Z = operators.spmatmul(X, Y)
        crp, cci, cva = api.bamg_step_spgemm(*csr_dev(X), *csr_dev(Y))
        assert np.array_equal(crp.cpu().numpy(), Z.indptr)
        assert np.array_equal(cci.cpu().numpy(), Z.indices)
        den = (abs(X) @ abs(Y)).tocsr()
        den.sort_indices()
        err = np.abs(cva.cpu().numpy() - Z.data) / np.maximum(den.data, 1e-300)
        assert err.max() <= 1e-12


def test_spgemm_exact_cancellation_keeps_slot(api):
    X = sp.csr_matrix(np.array([[1.0, 1.0, 0.0], [0.0, 2.0, 1.0]]))
    Y = sp.csr_matrix(np.array([[2.0], [-2.0], [4.0]]))
    crp, cci, cva = api.bamg_step_spgemm(*csr_dev(X), *csr_dev(Y))
    assert crp.cpu().tolist() == [0, 1, 2] and cci.cpu().tolist() == [0, 0]
    assert cva.cpu().tolist() == [0.0, 0.0]


def test_jacobi_divisor_matches_oracle(api):
    rng_ = np.random.default_rng(9)
    n = 700
    M = sp.random(n, n, density=0.01, random_state=11, format="csr")
    M.data = rng_.uniform(-1, 1, M.nnz)
    M = (M + sp.diags(rng_.uniform(-1, 2, n))).tocsr()      # about a third of the diagonal <= 0
    M.sort_indices()
    T = M.T.tocsr()
    T.sort_indices()
    want = 1.0 / operators.jacobi_divisor(M)
    dev = lambda a, t: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", t)
    dinv, ns = api.bamg_step_jacobi_divisor(dev(M.indptr, torch.int32), dev(M.indices, torch.int32),
                                            dev(M.data, torch.float64), dev(T.indptr, torch.int32),
                                            dev(T.data, torch.float64))
    assert ns == int((M.diagonal() <= 0).sum()) > 0
    assert np.allclose(dinv.cpu().numpy(), want, rtol=1e-15, atol=0)


# ------------------------------------------------------------------ A12
def _coarse_problem(n_side=12):
    from oracle import setup as S
    ch = cg.tandem(2 * n_side)
    H = S.bamg_setup(ch.csr(), S.Params(r=8, max_levels=2, coarse_min=1, seed=4), grid=(ch.nx, ch.ny))
    L = H.levels[-1]
    return L.B.toarray(), L.M.toarray(), L.N.toarray()


# sizes: 144 (own rows in shared memory), 289 (FP64 rows in global memory),
# 441 (both precisions in global memory), 9 (fewer rows than cluster blocks)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("side,r", [(12, 8), (17, 16), (21, 8), (3, 8)])
def test_coarsest_triplets_and_pinv(api, prec, side, r):
    Bd, Md, Nd = _coarse_problem(side)
    sig, U, V, Pinv = api.bamg_step_coarsest(Bd, Md, Nd, r, prec=prec)
    sig, U, V, Pinv = (t.cpu().numpy() for t in (sig, U, V, Pinv))
    so, Uo, Vo = coarsest.generalized_triplets(Bd, Md, Nd, r)
    Xo = coarsest.pinv_drop_smallest(Bd)
    scale = np.abs(Bd).max()
    if prec == "fp64":
        assert np.allclose(sig, so, rtol=1e-10, atol=1e-13 * scale)
        gaps = np.diff(np.concatenate([[0.0], so, [np.inf]]))
        for k in range(r):
            if min(gaps[k], gaps[k + 1]) < 1e-6 * scale:
                continue                          # clustered: vectors not unique
            tolv = 1e-12 * scale / min(gaps[k], gaps[k + 1]) * 100
            assert np.abs(V[:, k] - Vo[:, k]).max() <= tolv * np.abs(Vo[:, k]).max(), k
            assert np.abs(U[:, k] - Uo[:, k]).max() <= tolv * np.abs(Uo[:, k]).max(), k
        assert np.abs(Pinv - Xo).max() <= 1e-9 * np.abs(Xo).max()
    else:
        # FP32 bounds: the 1e-5 bar scaled by the conditioning the FP32 steps
        # see.  Singular values of the whitened C = L_M^-1 B L_N^-T move by at
        # most the norm of its backward error, which the triangular solves
        # scale by cond(L_M) + cond(L_N) = sqrt(cond M) + sqrt(cond N) (Weyl);
        # a singular vector moves by that over its gap; the Gauss-Jordan
        # inverse behind B^+ by cond(B + e e^T) relative.
        LM, LN = np.linalg.cholesky(Md), np.linalg.cholesky(Nd)
        C = np.linalg.solve(LM, np.linalg.solve(LN, Bd.T).T)
        cnorm = np.linalg.norm(C, 2)
        kap = np.sqrt(np.linalg.cond(Md)) + np.sqrt(np.linalg.cond(Nd))
        tau = 1e-5 * kap * cnorm
        assert np.abs(sig - so).max() <= tau, (np.abs(sig - so).max(), tau)
        gaps = np.diff(np.concatenate([[0.0], so, [np.inf]]))
        for k in range(1, r):
            g = min(gaps[k], gaps[k + 1])
            if g < 1e-3 * cnorm:
                continue                          # clustered: vectors not unique
            # whitened vectors: L_N^T v is unit, so the angle error is tau / gap
            # (in FP32 two entries of nearly equal magnitude may pick the
            # other sign; the FP64 comparison above checks the convention)
            ev = min(np.linalg.norm(LN.T @ (V[:, k] - Vo[:, k])), np.linalg.norm(LN.T @ (V[:, k] + Vo[:, k])))
            assert ev <= 10 * tau / g, (k, ev, tau / g)
        kb = np.linalg.cond(Bd + 1.0 / Bd.shape[0])
        assert np.abs(Pinv - Xo).max() <= 1e-5 * kb * np.abs(Xo).max(), (np.abs(Pinv - Xo).max(), kb)
    # residuals of the generalized singular equations (any precision); the
    # FP32 rounding error of the factorizations grows about linearly with n
    tol = 1e-11 if prec == "fp64" else max(1e-4, 1e-6 * Bd.shape[0])
    for k in range(r):
        assert np.linalg.norm(Bd @ V[:, k] - sig[k] * Md @ U[:, k]) <= tol * scale
        assert np.linalg.norm(Bd.T @ U[:, k] - sig[k] * Nd @ V[:, k]) <= tol * scale
