"""Solve phase: V-cycle preconditioner and GMRES variants (Section 6).

V-cycle (Section 3, eq. coarse_grid_correction / error_propagator_twogrid):
from z = 0, nu_pre Jacobi sweeps, residual, restriction with Q, recursive
coarse solve (pseudo-inverse on the coarsest level), interpolation with P,
nu_post Jacobi sweeps.  Started from zero it is the linear map z = C b.

Section 6 applies GMRES to the residual equation B e = -B x^(0)
(eq. residual).  The paper preconditions on the left (eq. prec_residual);
the GPU library uses flexible GMRES with the V-cycle on the right, which
also admits a preconditioner computed in lower precision.  Both are here,
with unpreconditioned GMRES(m) (Section 7 comparison) and two independent
reference solvers (dense null space, power iteration).

Stopping rule: the true ||B x||_1 / ||x||_1 of the current iterate.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import smoothing
from .setup import Hierarchy


def vcycle(H: Hierarchy, b: np.ndarray, l: int = 0) -> np.ndarray:
    p = H.params
    lev = H.levels[l]
    if l == len(H.levels) - 1:
        return H.Bpinv @ b
    z = np.zeros_like(b)
    for _ in range(p.nu_pre):
        z = smooth(H, lev, z, b)
    res = b - lev.B @ z
    z = z + lev.P @ vcycle(H, lev.Q @ res, l + 1)
    for _ in range(p.nu_post):
        z = smooth(H, lev, z, b)
    return z


def smooth(H: Hierarchy, lev, z: np.ndarray, b: np.ndarray) -> np.ndarray:
    """One sweep of the V-cycle smoother (Section 3): weighted Jacobi, or
    Gauss-Seidel (unweighted) in the level's row order with the Jacobi
    divisor d (b_ii where b_ii > 0)."""
    p = H.params
    if p.smoother == "jacobi":
        return z + p.omega * (b - lev.B @ z) / lev.d
    return smoothing.gauss_seidel(lev.B, z, b, lev.order, lev.d)


def rel_res_1(B, x):
    return np.abs(B @ x).sum() / np.abs(x).sum()


def _lsq_hessenberg(Hm: np.ndarray, beta: float) -> np.ndarray:
    g = np.zeros(Hm.shape[0])
    g[0] = beta
    return np.linalg.lstsq(Hm, g, rcond=None)[0]


def fgmres(B: sp.csr_matrix, x0: np.ndarray, precond, tol: float = 1e-10,
           restart: int = 20, max_iter: int = 1000):
    """Right-preconditioned flexible GMRES for B x = 0 from x0.

    Classical Gram-Schmidt with one re-orthogonalisation.  Returns
    (x, iterations, history of the true 1-norm ratio).
    """
    x = x0.copy()
    hist = [rel_res_1(B, x)]
    its = 0
    if hist[0] <= tol:
        return x, 0, hist
    n = x.shape[0]
    while its < max_iter:
        r = -(B @ x)
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        Hm = np.zeros((restart + 1, restart))
        V[0] = r / beta
        for j in range(restart):
            Z[j] = precond(V[j])
            w = B @ Z[j]
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            Hm[:j + 1, j] = h + h2
            Hm[j + 1, j] = np.linalg.norm(w)
            its += 1
            y = _lsq_hessenberg(Hm[:j + 2, :j + 1], beta)
            xj = x + Z[:j + 1].T @ y
            hist.append(rel_res_1(B, xj))
            if hist[-1] <= tol or Hm[j + 1, j] == 0.0 or its >= max_iter:
                return xj, its, hist
            V[j + 1] = w / Hm[j + 1, j]
        x = xj
    return x, its, hist


def gmres_left(B: sp.csr_matrix, x0: np.ndarray, precond, tol: float = 1e-10,
               restart: int = 50, max_iter: int = 1000):
    """GMRES on C B e = -C B x^(0) (eq. prec_residual), x = x^(0) + e.

    With precond = identity this is unpreconditioned GMRES(restart).
    """
    x = x0.copy()
    hist = [rel_res_1(B, x)]
    its = 0
    if hist[0] <= tol:
        return x, 0, hist
    n = x.shape[0]
    while its < max_iter:
        r = precond(-(B @ x))
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Hm = np.zeros((restart + 1, restart))
        V[0] = r / beta
        for j in range(restart):
            w = precond(B @ V[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            Hm[:j + 1, j] = h + h2
            Hm[j + 1, j] = np.linalg.norm(w)
            its += 1
            y = _lsq_hessenberg(Hm[:j + 2, :j + 1], beta)
            xj = x + V[:j + 1].T @ y
            hist.append(rel_res_1(B, xj))
            if hist[-1] <= tol or Hm[j + 1, j] == 0.0 or its >= max_iter:
                return xj, its, hist
            V[j + 1] = w / Hm[j + 1, j]
        x = xj
    return x, its, hist


def normalise_x(x: np.ndarray) -> np.ndarray:
    """Positive orientation and unit 1-norm (Section 2: x > 0 up to scale)."""
    return x / x.sum()


def bamg_solve(H: Hierarchy, tol: float = 1e-10, restart: int = 20,
               max_iter: int = 500, left: bool = False):
    """BAMG-preconditioned GMRES from the setup's x^(0) (Section 6)."""
    B = H.levels[0].B
    prec = lambda b: vcycle(H, b)
    if left:
        x, its, hist = gmres_left(B, H.x0, prec, tol, restart, max_iter)
    else:
        x, its, hist = fgmres(B, H.x0, prec, tol, restart, max_iter)
    return normalise_x(x), its, hist


def dense_nullvector(A_dense: np.ndarray) -> np.ndarray:
    """Stationary vector from the SVD of the dense B = I - A (small n)."""
    B = np.eye(A_dense.shape[0]) - A_dense
    _, _, Vt = np.linalg.svd(B)
    return normalise_x(Vt[-1])


def direct_nullvector(A: sp.csr_matrix) -> np.ndarray:
    """Stationary vector from its definition (Section 2: B x = 0, x > 0,
    sum 1) by one sparse LU solve: for an irreducible chain B = I - A has
    rank n - 1 and 1^T B = 0, so the last equation is implied by the others;
    replacing it by x_{n-1} = 1 (nonzero, since x > 0) gives a nonsingular
    system.  One step of iterative refinement, then the 1-norm scaling."""
    import scipy.sparse.linalg as spl
    A = sp.csr_matrix(A)
    n = A.shape[0]
    C = (sp.identity(n, format="csr") - A).tocoo()
    keep = C.row != n - 1
    K = sp.csc_matrix((np.concatenate([C.data[keep], [1.0]]),
                       (np.concatenate([C.row[keep], [n - 1]]), np.concatenate([C.col[keep], [n - 1]]))),
                      shape=(n, n))
    b = np.zeros(n)
    b[n - 1] = 1.0
    lu = spl.splu(K, permc_spec="MMD_AT_PLUS_A")
    x = lu.solve(b)
    x += lu.solve(b - K @ x)
    return normalise_x(x)


def power_iteration(A: sp.csr_matrix, tol: float = 1e-13, max_iter: int = 10 ** 6):
    """x <- (I + A) x / 2 (lazy chain, aperiodic), 1-norm normalised."""
    n = A.shape[0]
    x = np.full(n, 1.0 / n)
    for it in range(max_iter):
        y = 0.5 * (x + A @ x)
        y /= y.sum()
        if np.abs(y - x).sum() <= tol:
            return y, it + 1
        x = y
    return x, max_iter
