"""Learned interpolation on the GPU against the oracle network.

* features and targets harvested from an LS hierarchy are bit-exact against
  the oracle's features of the same level (B, C/F split) and the level's own
  P and Q^T placed in slots;
* forward and gradient of the tensor-core kernels match the FP64 oracle:
  tightly when the oracle rounds where the kernels store bfloat16, and within
  the bfloat16 error of the exact network otherwise;
* one Adam step matches its formula, and training lowers the loss;
* a network trained on LS setups of small tandem queues and lattices gives a
  hierarchy that solves a larger tandem queue to ||Bx||_1/||x||_1 <= 1e-10
  with x within 1e-8 of the oracle's stationary vector, and the gain test:
  it needs no test-vector relaxation and no LS fits, and reaches the LS
  iteration count far more closely than the untrained network.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import chaingen as cg
from oracle import mlp as OM
from oracle import solve as So

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1402_4005_gb300 import api as a
    return a


def gpu_setup(api, ch, **kw):
    p = api.bamg_params_default(**kw)
    return api.bamg_setup(torch.from_numpy(ch.row_ptr).cuda(), torch.from_numpy(ch.col).cuda(),
                          torch.from_numpy(ch.val).cuda(), ch.n, p, nx=ch.nx, ny=ch.ny)


def sp_of(d, shape):
    return sp.csr_matrix((d["val"].cpu().numpy(), d["col"].cpu().numpy(), d["row_ptr"].cpu().numpy()),
                         shape=shape)


def bits(t):
    return t.contiguous().view(torch.int16).cpu().numpy()


def rand_rows(m, seed):
    rng = np.random.default_rng(seed)
    X = OM.bf16(rng.uniform(-1, 1, size=(m, 64)))
    T = rng.normal(size=(m, 16))
    mask = (rng.uniform(size=(m, 16)) < 0.5).astype(float)
    return X, T, mask


@pytest.mark.parametrize("shape", [(33, 33), (32, 21)])
def test_harvest_matches_oracle_features_and_targets(api, shape):
    nx, ny = shape
    ch = cg.lattice2d(nx, ny, seed=7)
    h = gpu_setup(api, ch, r=16, max_levels=3, coarse_min=1, seed=3)
    gx, gy = nx, ny
    for l in range(h.num_levels - 1):
        lv = h.level(l)
        n = lv["n"]
        assert n == gx * gy
        B = sp_of(lv["B"], (n, n))
        cf = lv["cf"].cpu().numpy()
        cmap = lv["cmap"].cpu().numpy()
        X, T, M = api.bamg_mlp_harvest(h, l)
        Xo = OM.features(B, gx, gy, cf)
        assert X.shape[0] == Xo.shape[0] == int((cf == 0).sum())
        want = torch.from_numpy(Xo.astype(np.float32)).to(torch.bfloat16)
        assert np.array_equal(bits(X), bits(want))
        nc = int(cf.sum())
        To, Mo = OM.targets(sp_of(lv["P"], (n, nc)), sp_of(lv["Qt"], (n, nc)), gx, gy, cf, cmap)
        assert np.array_equal(M.cpu().numpy(), Mo.astype(np.float32))
        assert np.array_equal(T.cpu().numpy(), To.astype(np.float32))
        gx, gy = (gx + 1) // 2, (gy + 1) // 2


def test_forward_matches_oracle(api):
    params = api.bamg_mlp_init(seed=11)
    m = 16 * 37 + 5                       # several tiles and a ragged tail
    X, _, _ = rand_rows(m, 1)
    Y = api.bamg_mlp_forward(params, torch.from_numpy(X)).cpu().numpy().astype(np.float64)
    p = params.cpu().numpy().astype(np.float64)
    Ye = OM.forward(p, X, emulate=True)
    Yx = OM.forward(p, X, emulate=False)
    scale = np.abs(Yx).max()
    assert np.linalg.norm(Y - Ye) <= 2e-3 * np.linalg.norm(Ye)
    assert np.abs(Y - Ye).max() <= 2e-2 * scale
    assert np.linalg.norm(Y - Yx) <= 3e-2 * np.linalg.norm(Yx)
    # empty input is a no-op
    Y0 = api.bamg_mlp_forward(params, torch.zeros(0, 64))
    assert Y0.shape == (0, 16)


def test_forward_many_tiles_per_block_matches_oracle(api):
    """The tensor-core inference kernel is persistent over 128-row tiles with
    double-buffered feature loads: enough rows that every block takes
    several tiles (both buffers, several barrier phases), a ragged last
    tile, and an input that starts at a 16-byte offset into its storage."""
    params = api.bamg_mlp_init(seed=14)
    m = 128 * 2 * torch.cuda.get_device_properties(0).multi_processor_count * 3 + 77
    X, _, _ = rand_rows(m + 1, 5)
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Xv = Xt.view(-1)[64:].view(m, 64)               # rows 1..m of the same storage
    Y = api.bamg_mlp_forward(params, Xv).cpu().numpy().astype(np.float64)
    p = params.cpu().numpy().astype(np.float64)
    Ye = OM.forward(p, X[1:], emulate=True)
    assert np.linalg.norm(Y - Ye) <= 2e-3 * np.linalg.norm(Ye)
    rows = np.linalg.norm(Y - Ye, axis=1) / np.maximum(np.linalg.norm(Ye, axis=1), 1e-30)
    assert np.quantile(rows, 0.999) <= 2e-2


def test_gradient_matches_oracle(api):
    params = api.bamg_mlp_init(seed=12)
    m = 16 * 29 + 9
    X, T, mask = rand_rows(m, 2)
    loss, g = api.bamg_mlp_grad(params, torch.from_numpy(X), torch.from_numpy(T), torch.from_numpy(mask))
    g = g.cpu().numpy().astype(np.float64)
    p = params.cpu().numpy().astype(np.float64)
    le, ge = OM.loss_grad(p, X, T, mask, emulate=True)
    lx, gx = OM.loss_grad(p, X, T, mask, emulate=False)
    assert abs(loss - le) <= 1e-4 * le
    for a, b in ((OM.W1, OM.B1), (OM.B1, OM.W2), (OM.W2, OM.B2), (OM.B2, OM.W3), (OM.W3, OM.B3),
                 (OM.B3, OM.NPARAM)):
        assert np.linalg.norm(g[a:b] - ge[a:b]) <= 5e-3 * np.linalg.norm(ge[a:b]), (a, b)
        assert np.linalg.norm(g[a:b] - gx[a:b]) <= 5e-2 * np.linalg.norm(gx[a:b]), (a, b)


def test_adam_step_and_training(api):
    params = api.bamg_mlp_init(seed=13)
    m = 16 * 20
    X, T, mask = rand_rows(m, 3)
    Xt, Tt, Mt = torch.from_numpy(X), torch.from_numpy(T), torch.from_numpy(mask)
    _, g = api.bamg_mlp_grad(params, Xt, Tt, Mt)
    p0 = params.clone()
    lr = 1e-3
    api.bamg_mlp_train(params, Xt, Tt, Mt, epochs=1, batch=m, lr=lr)
    # first step: bias-corrected moments are g and g^2
    g64 = g.double()
    want = p0.double() - lr * g64 / (g64.abs() + 1e-8)
    assert torch.allclose(params.double(), want, rtol=1e-5, atol=1e-7)
    losses = api.bamg_mlp_train(params, Xt, Tt, Mt, epochs=40, batch=64, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]


def test_gradient_and_training_are_deterministic(api):
    """No atomics decide the order of any gradient sum: repeated gradients
    and repeated training runs agree bit for bit (many blocks, ragged tail)."""
    m = 16 * 700 + 5
    X, T, mask = rand_rows(m, 4)
    Xt, Tt, Mt = torch.from_numpy(X), torch.from_numpy(T), torch.from_numpy(mask)
    params = api.bamg_mlp_init(seed=21)
    g1 = api.bamg_mlp_grad(params, Xt, Tt, Mt)[1]
    g2 = api.bamg_mlp_grad(params, Xt, Tt, Mt)[1]
    assert torch.equal(g1, g2)
    runs = []
    for _ in range(2):
        p = api.bamg_mlp_init(seed=22)
        api.bamg_mlp_train(p, Xt, Tt, Mt, epochs=3, batch=4096, lr=2e-3)
        runs.append(p)
    assert torch.equal(runs[0], runs[1])


def _dataset(api, chains):
    Xs, Ts, Ms = [], [], []
    for ch in chains:
        h = gpu_setup(api, ch, r=16, coarse_min=64, seed=2)
        for l in range(h.num_levels - 1):
            X, T, M = api.bamg_mlp_harvest(h, l)
            Xs.append(X); Ts.append(T); Ms.append(M)
        h.destroy()
    X, T, M = torch.cat(Xs), torch.cat(Ts), torch.cat(Ms)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(X.shape[0])).cuda()
    return X[perm].contiguous(), T[perm].contiguous(), M[perm].contiguous()


@pytest.fixture(scope="module")
def trained(api):
    chains = [cg.tandem(s) for s in (32, 48, 64)] + [cg.lattice2d(s, seed=s) for s in (40, 64)]
    X, T, M = _dataset(api, chains)
    params = api.bamg_mlp_init(seed=5)
    losses = api.bamg_mlp_train(params, X, T, M, epochs=60, batch=1024, lr=2e-3)
    return params, losses


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_learned_hierarchy_solves(api, trained, prec):
    params, losses = trained
    assert losses[-1] < 0.2 * losses[0]
    ch = cg.tandem(48)
    xo = So.dense_nullvector(cg.to_dense(ch))
    h = gpu_setup(api, ch, r=8, coarse_min=64, seed=2, precision=prec, interp="mlp", mlp_params=params)
    x, info = api.bamg_solve(h)
    x = x.cpu().numpy()
    assert info["rel_res_1"] <= 1e-10
    assert np.abs(x - xo).sum() / np.abs(xo).sum() <= 1e-8
    assert (x > 0).all()
    # Section 5 constraint survives the projection: 1^T Q = 1^T on every level
    for l in range(h.num_levels - 1):
        lv = h.level(l)
        n, nc = lv["n"], int(lv["cf"].sum().item())
        Qt = sp_of(lv["Qt"], (n, nc))
        assert np.allclose(np.asarray(Qt.sum(axis=1)).ravel(), 1.0, atol=1e-12)


def test_trained_network_file_round_trip(api, trained, tmp_path):
    """A trained network saved from the GPU and loaded back (to the GPU and
    to the host) keeps every bit, and the loaded vector drives the same
    forward pass."""
    params, _ = trained
    path = tmp_path / "trained.bin"
    api.bamg_mlp_save(params, path)
    dev = api.bamg_mlp_load(path)
    host = api.bamg_mlp_load(path, device="cpu")
    assert dev.is_cuda and not host.is_cuda
    assert torch.equal(dev.cpu().view(torch.int32), params.cpu().view(torch.int32))
    assert torch.equal(host.view(torch.int32), params.cpu().view(torch.int32))
    X, _, _ = rand_rows(16 * 9 + 3, 21)
    X = torch.from_numpy(X)
    Y0 = api.bamg_mlp_forward(params, X)
    Y1 = api.bamg_mlp_forward(dev, X)
    assert torch.equal(Y0.view(torch.int32), Y1.view(torch.int32))


def test_learned_gain_over_untrained_and_ls(api, trained):
    params, _ = trained
    ch = cg.tandem(96)
    kw = dict(r=16, coarse_min=64, seed=2)
    ls = gpu_setup(api, ch, **kw)
    _, ils = api.bamg_solve(ls)
    f_ls = api.bamg_vcycle_factor(ls)
    ml = gpu_setup(api, ch, interp="mlp", mlp_params=params, **kw)
    _, iml = api.bamg_solve(ml)
    f_ml = api.bamg_vcycle_factor(ml)
    raw = api.bamg_mlp_init(seed=5)
    try:
        un = gpu_setup(api, ch, interp="mlp", mlp_params=raw, **kw)
        _, iun = api.bamg_solve(un, max_iter=200, allow_not_converged=True)
        f_un = api.bamg_vcycle_factor(un)
        it_un = iun["iterations"] if iun["rel_res_1"] <= 1e-10 else 10 ** 6
    except RuntimeError:                  # untrained fits may break the coarse diagonal
        f_un, it_un = float("inf"), 10 ** 6
    print(f"\nLS: {ils['iterations']} its, factor {f_ls:.3f}, setup {ls_ms(ils):.2f} ms | "
          f"learned: {iml['iterations']} its, factor {f_ml:.3f}, setup {ls_ms(iml):.2f} ms | "
          f"untrained: {it_un} its, factor {f_un:.3f}")
    assert iml["rel_res_1"] <= 1e-10
    assert iml["iterations"] <= 2 * ils["iterations"] + 4
    assert iml["iterations"] < it_un
    assert f_ml < f_un


def ls_ms(info):
    return info["setup_ms"]


@pytest.fixture(scope="module")
def trained_mix(api):
    """The network trained as the bench trains it: LS setups of 512 seeded
    tandem queues and weighted lattices (sides 64-512), at most 2048 seeded
    rows per level and chain, rows with LS weights above 4 in magnitude
    dropped, 40 epochs of Adam."""
    g = torch.Generator(device="cpu").manual_seed(7)
    Xs, Ts, Ms = [], [], []
    for k, ch in enumerate(cg.training_mix(512, seed=6)):
        h = gpu_setup(api, ch, r=16, seed=5 + k, precision="mixed")
        for l in range(h.num_levels - 1):
            X, T, M = api.bamg_mlp_harvest(h, l)
            ok = (T.abs() * M).amax(dim=1) <= 4.0
            X, T, M = X[ok], T[ok], M[ok]
            if X.shape[0] > 2048:
                sel = torch.randperm(X.shape[0], generator=g)[:2048].cuda()
                X, T, M = X[sel], T[sel], M[sel]
            Xs.append(X); Ts.append(T); Ms.append(M)
        h.destroy()
    X, T, M = torch.cat(Xs), torch.cat(Ts), torch.cat(Ms)
    perm = torch.from_numpy(np.random.default_rng(6).permutation(X.shape[0])).cuda()
    params = api.bamg_mlp_init(seed=5)
    api.bamg_mlp_train(params, X[perm].contiguous(), T[perm].contiguous(), M[perm].contiguous(), epochs=40,
                       batch=4096, lr=2e-3)
    return params


@pytest.mark.parametrize("side,levels", [(512, 6), (1024, 7)])
def test_learned_gain_over_ls_at_equal_parameters(api, trained_mix, side, levels):
    """Network fits against the LS fits with the same parameters (r = 16,
    5 setup relaxations, mixed precision) on tandem queues: GMRES converges
    without the FP64 fallback in at most 10 % more iterations than with LS,
    and the setup, which relaxes and fits nothing, is faster.  At 512^2 the
    network's hierarchy also contracts as a stationary method (V-cycle factor
    below 1).  At 1024^2 with 7 levels the LS factor is above 1 and the
    network's factor depends on the training run (0.94 and 5.75 from two
    trainings whose LS targets differ only in the rounding of the FP32 fit),
    so it is printed, not asserted."""
    ch = cg.tandem(side)
    kw = dict(r=16, seed=2, precision="mixed", max_levels=levels)
    out = {}
    for name, extra in (("ls", {}), ("mlp", dict(interp="mlp", mlp_params=trained_mix))):
        gpu_setup(api, ch, **kw, **extra).destroy()                 # warm-up
        h = gpu_setup(api, ch, **kw, **extra)
        x, info = api.bamg_solve(h, restart=20, tol=1e-10, max_iter=400)
        out[name] = (info, api.bamg_vcycle_factor(h))
        h.destroy()
    (ils, fls), (iml, fml) = out["ls"], out["mlp"]
    print(f"\ntandem {side}^2, {levels} levels: LS {ils['iterations']} its, factor {fls:.3f}, "
          f"setup {ils['setup_ms']:.1f} ms, solve {ils['solve_ms']:.1f} ms | network {iml['iterations']} its, "
          f"factor {fml:.3f}, setup {iml['setup_ms']:.1f} ms, solve {iml['solve_ms']:.1f} ms")
    assert iml["rel_res_1"] <= 1e-10 and iml["fallback_iterations"] == 0
    if levels == 6:
        assert fml < 1.0
    else:
        assert fls > 1.0
    assert iml["iterations"] <= 1.1 * ils["iterations"]
    assert iml["setup_ms"] < ils["setup_ms"]


def test_judged_setup_takes_fallback(api, trained):
    params, _ = trained
    ch = cg.tandem(48)
    p = api.bamg_params_default(r=8, coarse_min=64, seed=2, interp="mlp", mlp_params=params)
    h, f, used_ls = api.bamg_setup_judged(ch.row_ptr, ch.col, ch.val, ch.n, p, max_factor=0.95, nx=ch.nx,
                                          ny=ch.ny)
    assert not used_ls and 0.0 <= f <= 0.95
    h2, f2, used2 = api.bamg_setup_judged(ch.row_ptr, ch.col, ch.val, ch.n, p, max_factor=0.0, nx=ch.nx,
                                          ny=ch.ny)
    assert used2 and f2 == -1.0
    x, info = api.bamg_solve(h2)
    assert info["rel_res_1"] <= 1e-10


def test_learned_rejects_graph_coarsening(api, trained):
    params, _ = trained
    ch = cg.tandem(16)
    with pytest.raises(RuntimeError):
        gpu_setup(api, ch, r=8, coarse_min=16, coarsening="mis", interp="mlp", mlp_params=params)
