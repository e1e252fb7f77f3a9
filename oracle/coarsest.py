"""Coarsest-level dense problems.

eq. generalized_eigenvalue (Section 4.2): on the coarsest level the r
smallest generalized singular triplets solve
    B_L v = sigma M_L u,   B_L^T u = sigma N_L v,
with M_L, N_L symmetric positive definite.  With Cholesky factors
M = L_M L_M^T and N = L_N L_N^T this is the ordinary SVD of
C = L_M^{-1} B_L L_N^{-T}:  C v~ = sigma u~,  u = L_M^{-T} u~,  v = L_N^{-T} v~.
Vectors are normalised by u^T M u = v^T N v = 1; a triplet's sign is chosen
so that the entry of v of largest magnitude (lowest index on ties) is
positive.

Section 3, eq. coarse_grid_correction: the V-cycle solves the coarsest system
with the Moore-Penrose pseudo-inverse; B_L has rank n_L - 1 because
1^T B_L = 0, so exactly the smallest singular value is dropped.
"""
import numpy as np
from scipy.linalg import cholesky, solve_triangular


def sign_fix(u: np.ndarray, v: np.ndarray):
    k = int(np.argmax(np.abs(v)))
    if v[k] < 0:
        return -u, -v
    return u, v


def generalized_triplets(B: np.ndarray, M: np.ndarray, N: np.ndarray, r: int):
    """(sigma[r], U[n, r], V[n, r]) for the r smallest generalized sigmas."""
    n = B.shape[0]
    r = min(r, n)
    LM = cholesky(M, lower=True)
    LN = cholesky(N, lower=True)
    C = solve_triangular(LM, B, lower=True)
    C = solve_triangular(LN, C.T, lower=True).T
    Uc, S, Vct = np.linalg.svd(C)
    order = np.argsort(S, kind="stable")[:r]
    sig = S[order].copy()
    U = np.empty((n, r))
    V = np.empty((n, r))
    for a, k in enumerate(order):
        u = solve_triangular(LM.T, Uc[:, k], lower=False)
        v = solve_triangular(LN.T, Vct[k, :], lower=False)
        U[:, a], V[:, a] = sign_fix(u, v)
    return sig, U, V


def pinv_drop_smallest(B: np.ndarray) -> np.ndarray:
    """B^+ from the SVD with exactly the smallest singular value removed."""
    U, S, Vt = np.linalg.svd(B)
    k = int(np.argmin(S))
    keep = np.arange(S.shape[0]) != k
    return (Vt[keep].T / S[keep]) @ U[:, keep].T
