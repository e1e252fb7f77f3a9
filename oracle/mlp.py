"""Learned interpolation: plain FP64 statement of the network and its features.

TEST INFRASTRUCTURE ONLY (see the package header).  Not in the paper: a
small multilayer perceptron proposes, from the local stencil of B, the
weights that the least-squares fits of eq. ls_interpolation (P) and Section 5
(Q, columns summing to one) compute.  This module states, slowly and in
float64:

  features    the 64 inputs of a fine point of a geometric level
  slot        the neighbour-slot numbering shared by inputs and outputs
  targets     LS weights of a level placed in the 8 slots (with a mask)
  forward     the network 64 -> 64 -> 64 -> 16 with ReLU
  loss_grad   masked mean squared error and its gradient by backpropagation
  project_q   the shift of the Q outputs to sum one over J_i (Section 5)

Parameter vector layout (float): W1[64][64], b1[64], W2[64][64], b2[64],
W3[16][64], b3[16]; W[out][in].

``bf16`` rounds float32 values to bfloat16 (round to nearest, ties to even),
the input precision of the tensor-core products.  ``forward(...,
emulate=True)`` additionally rounds the two hidden activations (and, in the
gradient, the back-propagated errors) to bfloat16 where the GPU kernels
store them, so the two can be compared tightly; ``emulate=False`` is the
exact network.
"""
import numpy as np

F, H, O = 64, 64, 16
W1, B1 = 0, 64 * 64
W2, B2 = B1 + 64, B1 + 64 + 64 * 64
W3, B3 = B2 + 64, B2 + 64 + 16 * 64
NPARAM = B3 + 16


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    Rounds the float32 value of x: keep the upper 16 bits of its IEEE
    encoding after adding half an ulp of bfloat16 (0x7FFF) plus the lowest
    kept bit (ties to even)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    bits = a.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    """Weights and biases as float64 arrays from the flat parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    return (p[W1:B1].reshape(H, F), p[B1:W2], p[W2:B2].reshape(H, H), p[B2:W3],
            p[W3:B3].reshape(O, H), p[B3:NPARAM])


def slot(di: int, dj: int) -> int:
    """Slot of the neighbour at grid offset (di, dj) in the 3x3 box, counted
    row-major with the centre skipped: (-1,-1) -> 0 ... (1,1) -> 7."""
    s = (di + 1) * 3 + (dj + 1)
    assert s != 4
    return s - 1 if s > 4 else s


def features(B, nx: int, ny: int, cf) -> np.ndarray:
    """Inputs of the fine points (ascending state order) of a geometric level.

    B: scipy sparse n x n, state s = gx*ny + gy; cf: 1 = coarse.  Row of a
    fine point i: b_{i,i+o}/b_ii (25 offsets o of the 5x5 box, row-major),
    then b_{i+o,i}/b_ii, then the coarse indicators of the 8 neighbours of
    the 3x3 box, then a constant 1 and five zeros.  The ratio is formed in
    float64 as b * (1/b_ii), then rounded to float32 and to bfloat16."""
    B = B.tocsr()
    Bd = {}
    for i in range(B.shape[0]):
        for p in range(B.indptr[i], B.indptr[i + 1]):
            Bd[(i, int(B.indices[p]))] = float(B.data[p])
    fine = [i for i in range(nx * ny) if not cf[i]]
    X = np.zeros((len(fine), F))
    for row, i in enumerate(fine):
        gi, gj = divmod(i, ny)
        dii = Bd.get((i, i), 0.0)
        inv = 1.0 / dii if dii != 0.0 else 0.0
        k = 0
        for di in range(-2, 3):
            for dj in range(-2, 3):
                a, b = gi + di, gj + dj
                if 0 <= a < nx and 0 <= b < ny:
                    j = a * ny + b
                    X[row, k] = Bd.get((i, j), 0.0) * inv
                    X[row, 25 + k] = Bd.get((j, i), 0.0) * inv
                k += 1
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                if di == 0 and dj == 0:
                    continue
                a, b = gi + di, gj + dj
                if 0 <= a < nx and 0 <= b < ny and cf[a * ny + b]:
                    X[row, 50 + slot(di, dj)] = 1.0
        X[row, 58] = 1.0
    return bf16(X)


def targets(P, Qt, nx: int, ny: int, cf, cmap):
    """LS weights of a geometric level in the 8 slots: T (nF x 16: P then Q)
    and the mask of the slots that belong to J_i.  P, Qt: n x n_c sparse with
    the coarse index cmap[j] of state j."""
    n = nx * ny
    coarse_state = {int(cmap[j]): j for j in range(n) if cf[j]}
    P, Qt = P.tocsr(), Qt.tocsr()
    fine = [i for i in range(n) if not cf[i]]
    T = np.zeros((len(fine), O))
    M = np.zeros((len(fine), O))
    for row, i in enumerate(fine):
        gi, gj = divmod(i, ny)
        for X, off in ((P, 0), (Qt, 8)):
            for p in range(X.indptr[i], X.indptr[i + 1]):
                j = coarse_state[int(X.indices[p])]
                a, b = divmod(j, ny)
                s = slot(a - gi, b - gj)
                T[row, off + s] = X.data[p]
                M[row, off + s] = 1.0
    return T, M


def forward(params, X, emulate=False, cache=False):
    """The network on the rows of X: h1 = relu(W1 x + b1), h2 = relu(W2 h1 +
    b2), y = W3 h2 + b3.  Weights are taken at bfloat16 precision."""
    w1, b1, w2, b2, w3, b3 = unpack(params)
    w1, w2, w3 = bf16(w1), bf16(w2), bf16(w3)
    b1, b2, b3 = (np.asarray(b, dtype=np.float32).astype(np.float64) for b in (b1, b2, b3))
    rnd = bf16 if emulate else (lambda v: v)
    X = np.asarray(X, dtype=np.float64)
    h1 = rnd(np.maximum(X @ w1.T + b1, 0.0))
    h2 = rnd(np.maximum(h1 @ w2.T + b2, 0.0))
    y = h2 @ w3.T + b3
    if cache:
        return y, (X, h1, h2, w1, w2, w3)
    return y


def loss_grad(params, X, T, mask, emulate=False):
    """Loss sum(mask (y - t)^2) / sum(mask) and its gradient with respect to
    the parameter vector, by the chain rule layer by layer (backpropagation).

    With emulate=True the output error and the two back-propagated errors are
    rounded to bfloat16 before they enter the products, as in the kernels."""
    y, (X, h1, h2, w1, w2, w3) = forward(params, X, emulate=emulate, cache=True)
    T = np.asarray(T, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    count = mask.sum()
    inv = 1.0 / count if count > 0 else 0.0
    e = y - T
    loss = float((mask * e * e).sum() * inv)
    rnd = bf16 if emulate else (lambda v: v)
    d3 = 2.0 * mask * e * inv
    gb3 = d3.sum(0)
    d3r = rnd(d3)
    gw3 = d3r.T @ h2
    d2 = (d3r @ w3) * (h2 > 0)
    gb2 = d2.sum(0)
    d2r = rnd(d2)
    gw2 = d2r.T @ h1
    d1 = (d2r @ w2) * (h1 > 0)
    gb1 = d1.sum(0)
    d1r = rnd(d1)
    gw1 = d1r.T @ X
    g = np.zeros(NPARAM)
    g[W1:B1] = gw1.ravel()
    g[B1:W2] = gb1
    g[W2:B2] = gw2.ravel()
    g[B2:W3] = gb2
    g[W3:B3] = gw3.ravel()
    g[B3:NPARAM] = gb3
    return loss, g


def loss_exact(params, X, T, mask):
    """The loss of the exact network with weights used as given (no bfloat16
    rounding anywhere): the function that central differences check."""
    p = np.asarray(params, dtype=np.float64)
    w1, b1 = p[W1:B1].reshape(H, F), p[B1:W2]
    w2, b2 = p[W2:B2].reshape(H, H), p[B2:W3]
    w3, b3 = p[W3:B3].reshape(O, H), p[B3:NPARAM]
    h1 = np.maximum(X @ w1.T + b1, 0.0)
    h2 = np.maximum(h1 @ w2.T + b2, 0.0)
    y = h2 @ w3.T + b3
    count = mask.sum()
    return float((mask * (y - T) ** 2).sum() / count)


def grad_exact(params, X, T, mask):
    """Backpropagation of ``loss_exact`` (same rules as ``loss_grad`` with no
    rounding of weights or activations)."""
    p = np.asarray(params, dtype=np.float64)
    w1, b1 = p[W1:B1].reshape(H, F), p[B1:W2]
    w2, b2 = p[W2:B2].reshape(H, H), p[B2:W3]
    w3, b3 = p[W3:B3].reshape(O, H), p[B3:NPARAM]
    h1 = np.maximum(X @ w1.T + b1, 0.0)
    h2 = np.maximum(h1 @ w2.T + b2, 0.0)
    y = h2 @ w3.T + b3
    count = mask.sum()
    d3 = 2.0 * mask * (y - T) / count
    d2 = (d3 @ w3) * (h2 > 0)
    d1 = (d2 @ w2) * (h1 > 0)
    g = np.zeros(NPARAM)
    g[W1:B1] = (d1.T @ X).ravel()
    g[B1:W2] = d1.sum(0)
    g[W2:B2] = (d2.T @ h1).ravel()
    g[B2:W3] = d2.sum(0)
    g[W3:B3] = (d3.T @ h2).ravel()
    g[B3:NPARAM] = d3.sum(0)
    return g


def project_q(Y, J_slots):
    """P and Q weights of one fine point from its 16 outputs: the P weights
    of the slots in J_slots as predicted, the Q weights shifted by a common
    amount so that they sum to one (the constraint of Section 5)."""
    p = np.array([Y[s] for s in J_slots], dtype=np.float64)
    q = np.array([Y[8 + s] for s in J_slots], dtype=np.float64)
    if len(q):
        q = q + (1.0 - q.sum()) / len(q)
    return p, q
