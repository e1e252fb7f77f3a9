"""Least-squares interpolation P and constrained least-squares restriction Q.

Section 4.1, eq. ls_interpolation: for each fine variable i the row P_i
minimises  sum_k omega_k (v_i^(k) - sum_{j in J_i} p_ij v_j^(k))^2  over unit
test vectors v^(k), with weights omega_k = 1/||B v^(k)||^2 (eq. ls_weights).
Coarse rows of P are rows of the identity (eq. Pstructure).

Q is the transpose of an interpolation for B^T built from the left test
vectors u^(k) with weights 1/||B^T u^(k)||^2 (Section 4.1, last paragraph).
Section 5: u^(1) = 1 has infinite weight, so each column of Q must reproduce
1 exactly: the fit uses u^(2..r) subject to sum_j q_ji = 1.  The constrained
problem is solved by the null-space method (Golub-Van Loan): q = q0 + Z y with
q0 = 1/c and Z an orthonormal basis of the complement of 1.

Inputs are n x r blocks; ``s``/``t`` are the square roots of the weights for
*normalised* vectors, i.e. s_k = 1/||B v^(k)|| with ||v^(k)||_2 = 1.

Optional Tikhonov term (not in the paper, off by default): with ridge = delta
> 0 each fit also penalises lambda_i ||p - 1/c||^2, lambda_i = delta *
trace(G_i) / c, where G_i is the weighted Gram matrix of the c neighbour
columns and 1/c the equal weights of the simple-averaging operator of
Section 5.  delta = 0 is the paper's fit, delta -> infinity the averaging;
in between, only the directions the test vectors leave ill-determined (e.g.
the cross term of the four diagonal corners of a 2D centre point) are pulled
towards equal weights.  Solved as the augmented least-squares problem
[W^(1/2) X; sqrt(lambda) I] d = [W^(1/2)(y - X p0); 0], p = p0 + d.
"""
import numpy as np
import scipy.sparse as sp


def normalise(X: np.ndarray, cols=None) -> np.ndarray:
    """Scale the chosen columns to unit 2-norm (Section 4.1: ||v^(k)|| = 1)."""
    X = X.copy()
    cols = range(X.shape[1]) if cols is None else cols
    for k in cols:
        X[:, k] /= np.linalg.norm(X[:, k])
    return X


def weights(B: sp.csr_matrix, X: np.ndarray, cols=None) -> np.ndarray:
    """sqrt(omega_k) = 1/||B x^(k)||_2 for the chosen columns (eq. ls_weights)."""
    r = X.shape[1]
    cols = range(r) if cols is None else cols
    s = np.zeros(r)
    BX = B @ X
    for k in cols:
        s[k] = 1.0 / np.linalg.norm(BX[:, k])
    return s


def _assemble(n, nc, cf, cmap, J, rows_val) -> sp.csr_matrix:
    """CSR (fine rows, coarse columns): identity rows on C, fitted rows on F."""
    indptr = [0]
    idx = []
    val = []
    for i in range(n):
        if cf[i]:
            idx.append(int(cmap[i])); val.append(1.0)
        else:
            cols = [int(cmap[j]) for j in J[i]]
            idx.extend(cols); val.extend(rows_val[i])
        indptr.append(len(idx))
    M = sp.csr_matrix((np.array(val, dtype=np.float64), np.array(idx, dtype=np.int64),
                       np.array(indptr, dtype=np.int64)), shape=(n, nc))
    return M


def ridge_lambda(Vw: np.ndarray, ridge: float) -> float:
    """lambda_i = delta * trace(Vw^T Vw) / c (zero when the fit is plain)."""
    return ridge * float(np.sum(Vw * Vw)) / Vw.shape[1] if ridge > 0 else 0.0


def _ridge_lstsq(A: np.ndarray, b: np.ndarray, lam: float) -> np.ndarray:
    """argmin_d ||b - A d||^2 + lam ||d||^2 via the augmented system."""
    if lam <= 0:
        return np.linalg.lstsq(A, b, rcond=None)[0]
    m = A.shape[1]
    Aa = np.vstack([A, np.sqrt(lam) * np.eye(m)])
    ba = np.concatenate([b, np.zeros(m)])
    return np.linalg.lstsq(Aa, ba, rcond=None)[0]


def fit_row(Vw: np.ndarray, yw: np.ndarray, ridge: float = 0.0) -> np.ndarray:
    """argmin_p ||yw - Vw p||_2 (minimum-norm if rank deficient); with
    ridge > 0 plus lambda ||p - 1/c||^2."""
    if ridge <= 0:
        return np.linalg.lstsq(Vw, yw, rcond=None)[0]
    c = Vw.shape[1]
    p0 = np.full(c, 1.0 / c)
    return p0 + _ridge_lstsq(Vw, yw - Vw @ p0, ridge_lambda(Vw, ridge))


def fit_row_sum_one(Vw: np.ndarray, yw: np.ndarray, ridge: float = 0.0) -> np.ndarray:
    """argmin_q ||yw - Vw q||_2 subject to sum(q) = 1 (null-space method);
    with ridge > 0 plus lambda ||q - 1/c||^2 = lambda ||y||^2 (Z orthonormal)."""
    c = Vw.shape[1]
    if c == 1:
        return np.ones(1)
    q0 = np.full(c, 1.0 / c)
    Qf, _ = np.linalg.qr(np.ones((c, 1)), mode="complete")
    Z = Qf[:, 1:]
    y = _ridge_lstsq(Vw @ Z, yw - Vw @ q0, ridge_lambda(Vw, ridge))
    return q0 + Z @ y


def ls_interpolation(V: np.ndarray, s: np.ndarray, cf, cmap, J, ridge: float = 0.0) -> sp.csr_matrix:
    """P (n x n_c) from eq. ls_interpolation; V normalised, s = sqrt(omega)."""
    n = V.shape[0]
    nc = int(cf.sum())
    rows = {}
    for i, Ji in J.items():
        Vw = V[Ji, :].T * s[:, None]
        yw = V[i, :] * s
        rows[i] = fit_row(Vw, yw, ridge)
    return _assemble(n, nc, cf, cmap, J, rows)


def ls_restriction_T(U: np.ndarray, t: np.ndarray, cf, cmap, J, ridge: float = 0.0) -> sp.csr_matrix:
    """Q^T (n x n_c): rows are the columns of Q, fitted to u^(2..r) with the
    constraint that each sums to one (Section 5, eq. weight_infinity)."""
    n = U.shape[0]
    nc = int(cf.sum())
    rows = {}
    for i, Ji in J.items():
        Vw = U[Ji, 1:].T * t[1:, None]
        yw = U[i, 1:] * t[1:]
        rows[i] = fit_row_sum_one(Vw, yw, ridge)
    return _assemble(n, nc, cf, cmap, J, rows)


def averaging_restriction_T(cf, cmap, J, n) -> sp.csr_matrix:
    """Simple averaging (Section 5, the prior-work alternative): every entry
    of a column of Q equals 1/c, c = number of entries in that column."""
    rows = {i: np.full(len(Ji), 1.0 / len(Ji)) for i, Ji in J.items()}
    return _assemble(n, int(cf.sum()), cf, cmap, J, rows)
