"""Pins of the oracle's learned-interpolation network (CPU only).

The network is not in the paper, so the pins come from mathematics:
bfloat16 rounding against its definition and against PyTorch's conversion,
the analytic gradient against central differences of the loss, the affine
regime of the network against the composed matrix product, a constant
network in closed form, the feature layout on a uniform lattice whose
transition probabilities are known by hand, and the Section 5 constraint
after the Q projection.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import chaingen as cg
from oracle import mlp


def _rand_problem(rng, m=23):
    X = mlp.bf16(rng.uniform(-1, 1, size=(m, 64)))
    T = rng.normal(size=(m, 16))
    mask = (rng.uniform(size=(m, 16)) < 0.6).astype(float)
    params = np.zeros(mlp.NPARAM)
    params[mlp.W1:mlp.B1] = rng.uniform(-1, 1, 64 * 64) * np.sqrt(6 / 64)
    params[mlp.B1:mlp.W2] = rng.uniform(-0.1, 0.1, 64)
    params[mlp.W2:mlp.B2] = rng.uniform(-1, 1, 64 * 64) * np.sqrt(6 / 64)
    params[mlp.B2:mlp.W3] = rng.uniform(-0.1, 0.1, 64)
    params[mlp.W3:mlp.B3] = rng.uniform(-1, 1, 16 * 64) * np.sqrt(6 / 64)
    params[mlp.B3:] = rng.uniform(-0.1, 0.1, 16)
    return params, X, T, mask


def test_bf16_rounding_definition():
    # ulp of bfloat16 at 1 is 2^-7: halfway cases round to the even mantissa
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-1.0 / 3.0) == -0.333984375


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        rng.uniform(-2, 2, 5000)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def test_gradient_central_differences():
    rng = np.random.default_rng(1)
    params, X, T, mask = _rand_problem(rng)
    g = mlp.grad_exact(params, X, T, mask)
    idx = np.concatenate([rng.choice(np.arange(mlp.W1, mlp.B1), 40, replace=False),
                          np.arange(mlp.B1, mlp.B1 + 8),
                          rng.choice(np.arange(mlp.W2, mlp.B2), 40, replace=False),
                          np.arange(mlp.B2, mlp.B2 + 8),
                          rng.choice(np.arange(mlp.W3, mlp.B3), 40, replace=False),
                          np.arange(mlp.B3, mlp.NPARAM)])
    h = 1e-6
    fd = np.empty(len(idx))
    for t, k in enumerate(idx):
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        fd[t] = (mlp.loss_exact(pp, X, T, mask) - mlp.loss_exact(pm, X, T, mask)) / (2 * h)
    assert np.allclose(g[idx], fd, rtol=1e-5, atol=1e-8)


def test_rounded_gradient_equals_exact_on_representable_weights():
    # with bfloat16-representable weights and emulate=False the two
    # implementations compute the same function
    rng = np.random.default_rng(2)
    params, X, T, mask = _rand_problem(rng)
    for a, b in ((mlp.W1, mlp.B1), (mlp.W2, mlp.B2), (mlp.W3, mlp.B3)):
        params[a:b] = mlp.bf16(params[a:b])
    params = params.astype(np.float32).astype(np.float64)
    loss, g = mlp.loss_grad(params, X, T, mask)
    assert np.isclose(loss, mlp.loss_exact(params, X, T, mask), rtol=1e-12)
    assert np.allclose(g, mlp.grad_exact(params, X, T, mask), rtol=1e-10, atol=1e-14)


def test_affine_regime_is_the_composed_product():
    # positive weights, inputs and biases keep every ReLU active: the
    # network is y = W3 (W2 (W1 x + b1) + b2) + b3
    rng = np.random.default_rng(3)
    params = np.zeros(mlp.NPARAM)
    params[mlp.W1:mlp.B1] = mlp.bf16(rng.uniform(0, 0.1, 64 * 64))
    params[mlp.B1:mlp.W2] = 0.5
    params[mlp.W2:mlp.B2] = mlp.bf16(rng.uniform(0, 0.1, 64 * 64))
    params[mlp.B2:mlp.W3] = 0.25
    params[mlp.W3:mlp.B3] = mlp.bf16(rng.uniform(-1, 1, 16 * 64))
    params[mlp.B3:] = 0.125
    X = mlp.bf16(rng.uniform(0, 1, size=(9, 64)))
    w1, b1, w2, b2, w3, b3 = mlp.unpack(params)
    want = (w3 @ (w2 @ (w1 @ X.T + b1[:, None]) + b2[:, None]) + b3[:, None]).T
    assert np.allclose(mlp.forward(params, X), want, rtol=1e-13, atol=1e-13)


def test_constant_network_closed_form():
    rng = np.random.default_rng(4)
    params, X, T, mask = _rand_problem(rng)
    params[mlp.W3:mlp.B3] = 0.0
    c = np.linspace(-1, 1, 16).astype(np.float32).astype(np.float64)   # float32 biases
    params[mlp.B3:] = c
    y = mlp.forward(params, X)
    assert np.array_equal(y, np.broadcast_to(c, y.shape))
    loss, g = mlp.loss_grad(params, X, T, mask)
    cnt = mask.sum()
    assert np.isclose(loss, (mask * (c - T) ** 2).sum() / cnt, rtol=1e-13)
    assert np.allclose(g[mlp.B3:], 2 * (mask * (c - T)).sum(0) / cnt, rtol=1e-12, atol=1e-15)
    assert not g[mlp.W1:mlp.W3].any()        # no signal reaches the hidden layers


def test_features_of_a_uniform_lattice_point():
    ch = cg.uniform2d(5)
    A = ch.csr()
    B = (sp.identity(ch.n) - A).tocsr()
    cf = np.array([(s // 5) % 2 == 0 and (s % 5) % 2 == 0 for s in range(ch.n)], dtype=np.int8)
    X = mlp.features(B, 5, 5, cf)
    fine = [s for s in range(ch.n) if not cf[s]]
    x = X[fine.index(1 * 5 + 2)]          # grid point (1, 2)
    k = lambda di, dj: (di + 2) * 5 + (dj + 2)
    assert x[k(0, 0)] == 1.0 and x[25 + k(0, 0)] == 1.0
    # row: b_ij = -1/deg(j); (0,2) sits on the boundary (3 neighbours)
    assert x[k(-1, 0)] == mlp.bf16(-1 / 3)
    for o in ((1, 0), (0, -1), (0, 1)):
        assert x[k(*o)] == -0.25
    # column: b_ji = -1/deg(i) = -1/4 for the four neighbours
    for o in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        assert x[25 + k(*o)] == -0.25
    assert np.count_nonzero(x[:50]) == 10
    # coarse neighbours (0,2) and (2,2): slots 1 and 6
    assert list(np.flatnonzero(x[50:58])) == [1, 6]
    assert x[58] == 1.0 and not x[59:].any()


def test_slot_numbering():
    order = [(di, dj) for di in (-1, 0, 1) for dj in (-1, 0, 1) if (di, dj) != (0, 0)]
    assert [mlp.slot(*o) for o in order] == list(range(8))


def test_targets_place_weights_in_slots():
    # 3x3 grid, coarse corners; P of the centre (fine) point interpolates
    # from the 4 corners with weights 0.1..0.4, Q column with 0.25 each
    nx = ny = 3
    cf = np.array([1, 0, 1, 0, 0, 0, 1, 0, 1], dtype=np.int8)
    cmap = np.full(9, -1)
    cmap[[0, 2, 6, 8]] = np.arange(4)
    rows, cols, vals = [], [], []
    for c, s in enumerate([0, 2, 6, 8]):
        rows.append(s); cols.append(c); vals.append(1.0)
    for c, w in zip(range(4), (0.1, 0.2, 0.3, 0.4)):
        rows.append(4); cols.append(c); vals.append(w)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(9, 4))
    Qt = sp.csr_matrix(([1.0] * 4 + [0.25] * 4, (rows, cols)), shape=(9, 4))
    T, M = mlp.targets(P, Qt, nx, ny, cf, cmap)
    centre = [s for s in range(9) if not cf[s]].index(4)
    # corners of the 3x3 box: slots 0, 2, 5, 7
    assert np.allclose(T[centre, [0, 2, 5, 7]], [0.1, 0.2, 0.3, 0.4])
    assert np.allclose(T[centre, [8, 10, 13, 15]], 0.25)
    assert M[centre].sum() == 8 and M.sum() == 8


def test_q_projection_sums_to_one():
    rng = np.random.default_rng(5)
    for c in (1, 2, 4):
        Y = rng.normal(size=16)
        slots = sorted(rng.choice(8, c, replace=False))
        p, q = mlp.project_q(Y, slots)
        assert abs(q.sum() - 1.0) < 1e-14
        assert np.allclose(np.diff(q), np.diff(Y[[8 + s for s in slots]]))
        assert np.array_equal(p, Y[slots])
