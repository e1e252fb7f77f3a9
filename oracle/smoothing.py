"""Stationary smoothers (Section 3, eq. smoothing / error_propagator_smoothing).

Weighted Jacobi is the only smoother of the paper's experiments (Section 7:
omega = 0.7).  The paper writes its splitting as F = omega*D; the step that
converges for omega = 0.7 is x <- x + omega * D^{-1} (b - B x), i.e. the
splitting F = D / omega, and that is the reading used here.

Gauss-Seidel is one of the admissible splittings listed in Section 3.  It is
given here in the natural (lexicographic) order of the paper and in a
multicolour order (rows of one colour share no edge of the symmetrised graph
of B, so they can be updated together); Jacobi is order-independent, so its
multicolour schedule is the plain sweep.  The V-cycle takes either smoother
(Params.smoother); the setup relaxations stay weighted Jacobi.
"""
import numpy as np
import scipy.sparse as sp

from . import rng


def jacobi(B: sp.csr_matrix, d: np.ndarray, X: np.ndarray, rhs=None,
           omega: float = 0.7) -> np.ndarray:
    """One sweep X + omega * D^{-1} (rhs - B X); X may be a vector or n x r."""
    R = -(B @ X) if rhs is None else rhs - B @ X
    if X.ndim == 1:
        return X + omega * R / d
    return X + omega * R / d[:, None]


def gauss_seidel(B: sp.csr_matrix, x: np.ndarray, b: np.ndarray, order, d=None) -> np.ndarray:
    """One forward Gauss-Seidel sweep visiting the rows in ``order``:
    x_i <- x_i + (b_i - sum_j b_ij x_j) / d_i with the current x, which is
    (b_i - sum_{j != i} b_ij x_j) / b_ii for the default d_i = b_ii."""
    x = x.copy()
    if d is None:
        d = B.diagonal()
    for i in order:
        s = b[i]
        for p in range(B.indptr[i], B.indptr[i + 1]):
            s -= B.data[p] * x[B.indices[p]]
        x[i] = x[i] + s / d[i]
    return x


def greedy_colouring(B: sp.csr_matrix, Bt: sp.csr_matrix, key: np.ndarray) -> np.ndarray:
    """Colour = smallest colour not used by a neighbour coloured earlier,
    vertices visited by decreasing priority key (ties by index)."""
    n = B.shape[0]
    Bs = (abs(B) + abs(Bt)).tocsr()
    order = np.lexsort((np.arange(n), ~key))
    colour = np.full(n, -1, dtype=np.int64)
    for v in order:
        nb = Bs.indices[Bs.indptr[v]:Bs.indptr[v + 1]]
        used = set(int(c) for c in colour[nb] if c >= 0)
        c = 0
        while c in used:
            c += 1
        colour[v] = c
    return colour


def multicolour_order(colour: np.ndarray) -> np.ndarray:
    """Rows grouped by colour, ascending index inside each colour."""
    return np.lexsort((np.arange(colour.shape[0]), colour))


COLOUR_STREAM = 6144


def colouring_priorities(n: int, seed: int, level: int) -> np.ndarray:
    return rng.draw(seed, COLOUR_STREAM + level, n)


def level_colouring(B: sp.csr_matrix, Bt: sp.csr_matrix, seed: int, level: int) -> np.ndarray:
    """Greedy colouring of the symmetrised graph of level ``level`` with the
    SplitMix64 priorities of that level."""
    return greedy_colouring(B, Bt, colouring_priorities(B.shape[0], seed, level))
