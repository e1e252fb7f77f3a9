"""The optional Tikhonov term of the least-squares fits (bamg_params.ls_ridge,
not in the paper) against the oracle's option of the same name.

Runs after the core parity suites.  Per kernel: P rows and Q columns with
delta = 0.03 and 1.0, FP64 and FP32 test vectors, geometric and graph sets,
at 1e-12 (FP64) / 1e-5 (FP32) times 10 x the condition number of the
penalised system.  End to end: the uniform walk on a 129 x 129 grid with
r = 8 and up to four interpolation points (the Table uniform2d setting, where
the plain fit loses diagonal dominance on the coarse levels) and a Delaunay
walk with 3 to 8 interpolation points: C/F structure and patterns bit for
bit, values at 1e-8 (FP64) / 2e-3 (mixed), and a solve to
||Bx||_1/||x||_1 <= 1e-10 (1e-11 on the Delaunay walk, whose slower mixing
needs it) within 1e-8 of the closed form.
"""
import numpy as np
import pytest

import chaingen as cg
from oracle import coarsening, interp, operators, rng, smoothing
from oracle import setup as S
from oracle import solve as So

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


def smoothed(B, d, n, r, ld, seed, first_ones=False):
    X = np.zeros((n, ld))
    for k in range(r):
        X[:, k] = rng.uniform_pm1(seed, 2 * k, n)
    if first_ones:
        X[:, 0] = 1.0
    for _ in range(5):
        Y = smoothing.jacobi(B, d, X, None, 0.7)
        if first_ones:
            Y[:, 0] = 1.0
        X = Y
    return X


def sets_csr(J, cf, n):
    rp = [0]
    ci = []
    for i in range(n):
        if not cf[i]:
            ci.extend(J[i])
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32)


def penalised_cond(Xw, delta):
    c = Xw.shape[1]
    lam = delta * float(np.sum(Xw * Xw)) / c
    return np.linalg.cond(np.vstack([Xw, np.sqrt(lam) * np.eye(c)]))


@pytest.mark.parametrize("delta", [0.03, 1.0])
@pytest.mark.parametrize("geom,ld,r", [(True, 8, 8), (False, 16, 16)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_penalised_fits_against_oracle(api, geom, ld, r, prec, delta):
    if geom:
        ch = cg.uniform2d(31)
        B = operators.build_B(ch.csr())
        cf, cmap, _ = coarsening.geometric(31, 31)
        J = coarsening.geometric_sets(31, 31, cf)
    else:
        ch = cg.delaunay_walk(2500, seed=8)
        B = operators.build_B(ch.csr())
        Bt0 = operators.transpose(B)
        cf, cmap = coarsening.greedy_mis(B, Bt0, 2, 0)
        J = coarsening.graph_sets(B, Bt0, cf, 3, 8)
    n = ch.n
    Bt = operators.transpose(B)
    d = operators.diag(B)
    V = interp.normalise(smoothed(B, d, n, r, ld, 5)[:, :r])
    U = interp.normalise(smoothed(Bt, d, n, r, ld, 6, first_ones=True)[:, :r], range(1, r))
    s = interp.weights(B, V)
    t = interp.weights(Bt, U, range(1, r))
    P = interp.ls_interpolation(V, s, cf, cmap, J, ridge=delta)
    Qt = interp.ls_restriction_T(U, t, cf, cmap, J, ridge=delta)
    jrp, jci = sets_csr(J, cf, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Vp = np.zeros((n, ld)); Vp[:, :r] = V
    Up = np.zeros((n, ld)); Up[:, :r] = U
    sp_ = np.zeros(ld); sp_[:r] = s
    tp_ = np.zeros(ld); tp_[:r] = t
    fitP, rk1 = api.bamg_step_ls_fit(dev(jrp), dev(jci), dev(Vp).to(dt), sp_, r, ridge=delta)
    fitQ, rk2 = api.bamg_step_ls_fit(dev(jrp), dev(jci), dev(Up).to(dt), tp_, r, constrained=True, ridge=delta)
    fitP, fitQ = fitP.cpu().numpy(), fitQ.cpu().numpy()
    assert rk1 == 0 and rk2 == 0
    base = 1e-12 if prec == "fp64" else 1e-5
    for i in range(n):
        if cf[i]:
            continue
        a, b = jrp[i], jrp[i + 1]
        cols = cmap[J[i]]
        kp = penalised_cond(V[J[i], :].T * s[:, None], delta)
        pr = P[i, cols].toarray().ravel()
        assert np.abs(fitP[a:b] - pr).max() <= base * kp * 10 * max(1.0, np.abs(pr).max()), (i, kp)
        kq = penalised_cond(U[J[i], 1:].T * t[1:, None], delta)
        qr = Qt[i, cols].toarray().ravel()
        assert np.abs(fitQ[a:b] - qr).max() <= base * kq * 10 * max(1.0, np.abs(qr).max()), (i, kq)
        assert abs(fitQ[a:b].sum() - 1.0) <= 1e-13 * len(J[i])


def test_negative_weight_is_rejected(api):
    from paper_1402_4005_gb300._lib import BamgError
    ch = cg.uniform2d(9)
    p = api.bamg_params_default(r=8, max_levels=2, coarse_min=1, ls_ridge=-0.5)
    with pytest.raises(BamgError) as e:
        api.bamg_setup(dev(ch.row_ptr), dev(ch.col), dev(ch.val), ch.n, p, nx=9, ny=9)
    assert e.value.status == 1


def compare_hierarchies(h, H, vtol):
    assert h.num_levels == len(H.levels)
    for l, lev in enumerate(H.levels):
        g = h.level(l)
        assert g["n"] == lev.n
        names = [("B", lev.B)]
        if l < len(H.levels) - 1:
            names += [("P", lev.P), ("Qt", lev.Qt)]
            assert np.array_equal(g["cf"].cpu().numpy().astype(bool), lev.cf), l
        for nm, M in names:
            rp, ci, va = (g[nm]["row_ptr"].cpu().numpy(), g[nm]["col"].cpu().numpy(), g[nm]["val"].cpu().numpy())
            assert np.array_equal(rp, M.indptr), (l, nm)
            assert np.array_equal(ci, M.indices), (l, nm)
            err = np.abs(va - M.data).max() / np.abs(M.data).max()
            assert err <= vtol, (l, nm, err)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uniform_walk_129_with_penalty(api, prec):
    ch = cg.uniform2d(129)
    kw = dict(r=8, coarse_min=17 * 17, c_max=4, seed=2)
    p = api.bamg_params_default(precision=prec, ls_ridge=0.03, **kw)
    h = api.bamg_setup(dev(ch.row_ptr), dev(ch.col), dev(ch.val), ch.n, p, nx=129, ny=129)
    H = S.bamg_setup(ch.csr(), S.Params(ls_ridge=0.03, **kw), grid=(129, 129))
    compare_hierarchies(h, H, 1e-8 if prec == "fp64" else 2e-3)
    assert min(float(l.B.diagonal().min()) for l in H.levels) > 0
    x, info = api.bamg_solve(h, restart=20, tol=1e-10)
    x = x.cpu().numpy()
    xs = ch.meta["wdeg"] / ch.meta["wdeg"].sum()
    assert info["rel_res_1"] <= 1e-10
    assert np.abs(x - xs).sum() <= 1e-8
    _, its, _ = So.bamg_solve(H, tol=1e-10, restart=20)
    assert abs(info["iterations"] - its) <= (1 if prec == "fp64" else 3)


def test_delaunay_three_to_eight_points_with_penalty(api):
    ch = cg.delaunay_walk(8192, seed=3)
    kw = dict(r=16, coarse_min=200, coarsening="mis", c_min=3, c_max=8, nu_pre=5, nu_post=5, seed=3)
    p = api.bamg_params_default(ls_ridge=0.03, **kw)
    h = api.bamg_setup(dev(ch.row_ptr), dev(ch.col), dev(ch.val), ch.n, p)
    H = S.bamg_setup(ch.csr(), S.Params(ls_ridge=0.03, **kw))
    compare_hierarchies(h, H, 1e-8)
    x, info = api.bamg_solve(h, restart=30, tol=1e-11)
    xs = ch.meta["deg"] / ch.meta["deg"].sum()
    assert info["rel_res_1"] <= 1e-11
    assert np.abs(x.cpu().numpy() - xs).sum() <= 1e-8


def test_second_cycle_with_penalty_on_paper_tandem(api):
    """BAMG^2 with the penalised fits on the tandem queue with the paper's
    rates (Table tandem setting, 129^2 states): hierarchy of the second cycle
    against the oracle, solve within 1e-8 of the oracle's stationary vector,
    and fewer iterations than one cycle needs."""
    ch = cg.tandem(129, lam=11 / 31, mu1=10 / 31, mu2=10 / 31)
    kw = dict(r=8, coarse_min=17 * 17, c_max=4, seed=2)
    its = []
    for cycles in (1, 2):
        p = api.bamg_params_default(ls_ridge=0.03, setup_cycles=cycles, **kw)
        h = api.bamg_setup(dev(ch.row_ptr), dev(ch.col), dev(ch.val), ch.n, p, nx=129, ny=129)
        H = S.bamg_setup(ch.csr(), S.Params(ls_ridge=0.03, cycles=cycles, **kw), grid=(129, 129))
        compare_hierarchies(h, H, 1e-8)
        x, info = api.bamg_solve(h, restart=20, tol=1e-10)
        xo, _, _ = So.bamg_solve(H, tol=1e-12, restart=20)
        assert info["rel_res_1"] <= 1e-10
        assert np.abs(x.cpu().numpy() - xo).sum() <= 1e-8
        its.append(info["iterations"])
    assert its[1] < its[0], its
