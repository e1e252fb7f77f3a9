"""Multicolour Gauss-Seidel (the Gauss-Seidel splitting of Section 3 in a
multicolour order) against the oracle.

Colours and the rows-by-colour order are integer work and compared bit for
bit; a sweep is compared at 1e-12 relative (FP64) and 1e-5 (FP32); V-cycles
with the Gauss-Seidel smoother at the V-cycle tolerances of the solve tests;
a solve must reach ||Bx||_1/||x||_1 <= 1e-10 with x within 1e-8 of the
oracle's.
"""
import numpy as np
import pytest

import chaingen as cg
from oracle import operators, rng, smoothing
from oracle import setup as S
from oracle import solve as So

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api as a
    return a


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def graphs():
    return [("tandem33", cg.tandem(33)), ("lattice40", cg.lattice2d(40, seed=4)),
            ("delaunay5000", cg.delaunay_walk(5000, seed=6))]


@pytest.mark.parametrize("name,ch", graphs())
def test_colouring_and_row_order_match_oracle(api, name, ch):
    B = operators.build_B(ch.csr())
    Bt = operators.transpose(B)
    for seed, level in ((3, 0), (11, 2)):
        col, nc = api.bamg_step_colour(dev(B.indptr.astype(np.int32)), dev(B.indices.astype(np.int32)),
                                       dev(Bt.indptr.astype(np.int32)), dev(Bt.indices.astype(np.int32)), seed, level)
        want = smoothing.level_colouring(B, Bt, seed, level)
        got = col.cpu().numpy()
        assert np.array_equal(got, want), name
        assert nc == int(want.max()) + 1
        crp, rows = api.bamg_step_colour_rows(col, nc)
        assert np.array_equal(rows.cpu().numpy(), smoothing.multicolour_order(want))
        assert np.array_equal(np.diff(crp), np.bincount(want, minlength=nc))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sweep_matches_oracle(api, prec):
    ch = cg.delaunay_walk(3000, seed=2)
    B = operators.build_B(ch.csr())
    Bt = operators.transpose(B)
    d = operators.jacobi_divisor(B)
    x = rng.uniform_pm1(4, 1, ch.n)
    b = rng.uniform_pm1(4, 2, ch.n)
    want = smoothing.gauss_seidel(B, x, b, smoothing.multicolour_order(smoothing.level_colouring(B, Bt, 5, 1)), d)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rp, ci = dev(B.indptr.astype(np.int32)), dev(B.indices.astype(np.int32))
    col, nc = api.bamg_step_colour(rp, ci, dev(Bt.indptr.astype(np.int32)), dev(Bt.indices.astype(np.int32)), 5, 1)
    crp, rows = api.bamg_step_colour_rows(col, nc)
    xg = dev(x).to(dt)
    api.bamg_step_mcgs_sweep(rp, ci, dev(B.data).to(dt), dev(1.0 / d).to(dt), crp, rows, dev(b).to(dt), xg)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.abs(xg.double().cpu().numpy() - want).max() <= tol * np.abs(want).max()


def setup_pair(api, ch, prec, **kw):
    p = api.bamg_params_default(smoother="mcgs", precision=prec, **kw)
    h = api.bamg_setup(dev(ch.row_ptr), dev(ch.col), dev(ch.val), ch.n, p, nx=ch.nx, ny=ch.ny)
    H = S.bamg_setup(ch.csr(), S.Params(smoother="mcgs", **kw), grid=(ch.nx, ch.ny) if ch.nx else None)
    return h, H


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vcycle_with_gauss_seidel_matches_oracle(api, prec):
    """Colours of every smoothed level bit-exact; the V-cycle at 1e-7
    (FP64) / 1e-3 (FP32) of the oracle's, with odd and even sweep counts."""
    ch = cg.tandem(40)
    for nu in ((3, 3), (2, 1)):
        kw = dict(r=8, max_levels=3, coarse_min=1, seed=3, nu_pre=nu[0], nu_post=nu[1])
        h, H = setup_pair(api, ch, prec, **kw)
        for l, lev in enumerate(H.levels[:-1]):
            g = h.level(l)
            assert np.array_equal(g["colour"].cpu().numpy(), lev.colour), l
            assert g["ncolours"] == int(lev.colour.max()) + 1
        b = H.levels[0].B @ rng.uniform_pm1(5, 0, ch.n)
        z = h.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
        zo = So.vcycle(H, b)
        tol = 1e-7 if prec == "fp64" else 1e-3
        assert np.abs(z - zo).max() <= tol * np.abs(zo).max(), nu


def test_solve_with_gauss_seidel(api):
    ch = cg.tandem(48)
    kw = dict(r=8, max_levels=3, coarse_min=1, seed=2)
    h, H = setup_pair(api, ch, "mixed", **kw)
    x, info = api.bamg_solve(h, restart=20, tol=1e-10)
    assert info["rel_res_1"] <= 1e-10
    xo, _, _ = So.bamg_solve(H, tol=1e-12, restart=20)
    assert np.abs(x.cpu().numpy() - xo).sum() <= 1e-8


def test_batches_reject_gauss_seidel(api):
    from paper_1402_4005_gb300._lib import BamgError
    ch = cg.tandem(16)
    p = api.bamg_params_default(smoother="mcgs", r=8, max_levels=2, coarse_min=1)
    with pytest.raises(BamgError) as e:
        api.bamg_setup_batched([(ch.row_ptr, ch.col, ch.val, ch.n, ch.nx, ch.ny)], p)
    assert e.value.status == 9
