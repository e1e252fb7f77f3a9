"""Operators of the method: B = I - A, transposes and structural products.

Section 2 (eq. steadystatesystemlinear): B = I - A for a column-stochastic A.
Section 3: the coarse operator is the Petrov-Galerkin product B_c = Q B P;
Algorithm 1 also forms M_{l+1} = Q M_l Q^T and N_{l+1} = P^T N_l P.

Sparsity conventions: CSR, column indices ascending, and every product keeps
its *structural* pattern (the pattern of |X||Y|), including entries whose
value cancels to zero.
"""
import numpy as np
import scipy.sparse as sp


def validate_stochastic(A: sp.csr_matrix, tol: float = 1e-12):
    """Section 2: a_ij >= 0 and every column sum equals one."""
    if A.nnz and A.data.min() < 0:
        raise ValueError("negative transition probability")
    cs = np.asarray(A.sum(axis=0)).ravel()
    bad = np.abs(cs - 1.0) > tol
    if bad.any():
        raise ValueError(f"column {int(np.argmax(bad))} sums to {cs[bad][0]!r}")


def build_B(A: sp.csr_matrix) -> sp.csr_matrix:
    """B = I - A with the diagonal always stored (structural pattern of A + I)."""
    A = A.tocoo()
    n = A.shape[0]
    rows = np.concatenate([A.row, np.arange(n)])
    cols = np.concatenate([A.col, np.arange(n)])
    vals = np.concatenate([-A.data, np.ones(n)])
    B = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    B.sum_duplicates()
    B.sort_indices()
    return B


def diag(B: sp.csr_matrix) -> np.ndarray:
    return B.diagonal().copy()


def jacobi_divisor(B: sp.csr_matrix) -> np.ndarray:
    """Divisors d of the weighted Jacobi step x + omega D^{-1}(b - B x)
    (Section 3).  d_i = b_ii where b_ii > 0.  The paper does not treat a
    coarse operator Q B P with b_ii <= 0, where its step is undefined; there
    d_i is the larger of the l1 norms of row i and of column i of B (an
    l1-Jacobi row that serves the relaxations with B and with B^T).  A row
    and column that are both zero make the level unusable (ValueError)."""
    d = B.diagonal().copy()
    A = abs(B).tocsr()
    l1 = np.maximum(np.asarray(A.sum(axis=1)).ravel(), np.asarray(A.sum(axis=0)).ravel())
    bad = ~(d > 0)
    if np.any(bad & ~(l1 > 0)):
        raise ValueError("a row and column of B are zero")
    d[bad] = l1[bad]
    return d


def transpose(X: sp.csr_matrix) -> sp.csr_matrix:
    T = X.T.tocsr()
    T.sort_indices()
    return T


def _indicator(X: sp.csr_matrix) -> sp.csr_matrix:
    return sp.csr_matrix((np.ones_like(X.data), X.indices, X.indptr),
                         shape=X.shape)


def spmatmul(X: sp.csr_matrix, Y: sp.csr_matrix) -> sp.csr_matrix:
    """Z = X Y on the structural pattern of |X||Y| (no cancellation drops).

    The pattern comes from the product of the 0/1 indicator matrices (sums of
    positive numbers cannot vanish); the values come from the library product
    and are placed on that pattern (0 where the values cancelled exactly).
    """
    S = (_indicator(X) @ _indicator(Y)).tocsr()
    S.sort_indices()
    V = (X @ Y).tocsr()
    V.sort_indices()
    coo = S.tocoo()
    vals = np.asarray(V[coo.row, coo.col]).ravel().astype(np.float64)
    Z = sp.csr_matrix((vals, S.indices.copy(), S.indptr.copy()), shape=S.shape)
    return Z


def galerkin(Q: sp.csr_matrix, B: sp.csr_matrix, P: sp.csr_matrix) -> sp.csr_matrix:
    """B_c = Q B P (Section 3; Algorithm 1 'Compute B_{l+1} = Q_l B_l P_l')."""
    return spmatmul(Q, spmatmul(B, P))
