"""Stationary smoothers (Section 3, eq. smoothing / error_propagator_smoothing).

Weighted Jacobi is the only smoother of the paper's experiments (Section 7:
omega = 0.7).  The paper writes its splitting as F = omega*D; the step that
converges for omega = 0.7 is x <- x + omega * D^{-1} (b - B x), i.e. the
splitting F = D / omega, and that is the reading used here.

Gauss-Seidel is one of the admissible splittings listed in Section 3.  It is
given here in the natural (lexicographic) order of the paper and in a
multicolour order; Jacobi is order-independent, so its multicolour schedule
is the plain sweep.
"""
import numpy as np
import scipy.sparse as sp


def jacobi(B: sp.csr_matrix, d: np.ndarray, X: np.ndarray, rhs=None,
           omega: float = 0.7) -> np.ndarray:
    """One sweep X + omega * D^{-1} (rhs - B X); X may be a vector or n x r."""
    R = -(B @ X) if rhs is None else rhs - B @ X
    if X.ndim == 1:
        return X + omega * R / d
    return X + omega * R / d[:, None]


def gauss_seidel(B: sp.csr_matrix, x: np.ndarray, b: np.ndarray, order) -> np.ndarray:
    """One forward Gauss-Seidel sweep visiting the rows in ``order``."""
    x = x.copy()
    for i in order:
        s = b[i]
        dii = 0.0
        for p in range(B.indptr[i], B.indptr[i + 1]):
            j = B.indices[p]
            if j == i:
                dii = B.data[p]
            else:
                s -= B.data[p] * x[j]
        x[i] = s / dii
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
