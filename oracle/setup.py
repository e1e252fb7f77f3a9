"""Algorithm 1 (bamg_mle): the first bootstrap setup cycle.

Per level l (finest l = 0), top-down:
  * relax the test vectors: V with B_l, U with B_l^T, right-hand side 0
    (Algorithm 1, first smoothing loop); u^(1) = 1 is the exact left null
    vector (Section 5) and is kept fixed;
  * normalise to unit 2-norm and take sqrt-weights 1/||B v||, 1/||B^T u||
    (eq. ls_weights);
  * split C/F, choose J_i, fit P rows (eq. ls_interpolation) and Q columns
    (Section 5 constraint);
  * B_{l+1} = Q B_l P,  M_{l+1} = Q M_l Q^T,  N_{l+1} = P^T N_l P;
  * inject U, V to the coarse level (R = canonical injection).
On the coarsest level the r smallest generalized singular triplets are
computed (eq. generalized_eigenvalue).  Bottom-up, each level receives
(sigma, Q^T u_c, P v_c) and relaxes the inhomogeneous systems
B_l v = sigma M_l u and B_l^T u = sigma N_l v, both from the previous
iterates, then updates sigma by the generalized Rayleigh quotient
(eq. singular_value).

Subsequent cycles (Section 4, after Algorithm 1; the BAMG^2 rows of the
tables in Section 7) rebuild the hierarchy from the finest level with the
previous cycle's finest triplets as test vectors; their first smoothing on
every level is the inhomogeneous one with the sigma update, instead of the
homogeneous one.

Readings where the paper is silent: 5 setup relaxations per level and phase
(with 3, the r = 8 fits over-fit rough vectors and the first hierarchy can
diverge as a stationary method); the inner loop runs once (mu = 1);
x^(0) is the finest v of smallest sigma, scaled to a positive unit 1-norm.
Option ls_ridge (default 0, the paper's plain fit): a Tikhonov term that
pulls ill-determined directions of each LS fit towards equal weights
(see oracle.interp).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import coarsening, coarsest, interp, operators, rng, smoothing


@dataclass
class Params:
    r: int = 8
    max_levels: int = 25
    coarse_min: int = 300
    nu_setup: int = 5
    nu_pre: int = 3
    nu_post: int = 3
    omega: float = 0.7
    coarsening: str = "geometric"     # or "mis"
    c_min: int = 1
    c_max: int = 4
    seed: int = 1
    restriction: str = "ls"           # or "average" (Section 5 comparison)
    cycles: int = 1                   # bootstrap setup cycles (2 = BAMG^2)
    smoother: str = "jacobi"          # V-cycle smoother: "jacobi", "mcgs" or "gs" (natural order)
    ls_ridge: float = 0.0             # Tikhonov weight delta of the LS fits (0 = the paper's plain fit)


@dataclass
class Level:
    n: int
    B: sp.csr_matrix
    Bt: sp.csr_matrix
    d: np.ndarray
    M: sp.csr_matrix | None = None     # None = identity (finest level)
    N: sp.csr_matrix | None = None
    grid: tuple | None = None
    cf: np.ndarray | None = None
    cmap: np.ndarray | None = None
    J: dict | None = None
    P: sp.csr_matrix | None = None
    Qt: sp.csr_matrix | None = None
    Q: sp.csr_matrix | None = None
    s: np.ndarray | None = None
    t: np.ndarray | None = None
    colour: np.ndarray | None = None   # multicolour Gauss-Seidel: colours and row order
    order: np.ndarray | None = None


@dataclass
class Hierarchy:
    params: Params
    levels: list = field(default_factory=list)
    Bpinv: np.ndarray | None = None
    sigma: np.ndarray | None = None
    U: np.ndarray | None = None
    V: np.ndarray | None = None
    x0: np.ndarray | None = None

    def op_complexity(self) -> float:
        """eq. operator_complexity_def."""
        return sum(l.B.nnz for l in self.levels) / self.levels[0].B.nnz

    def grid_complexity(self) -> float:
        """Section 7: o_g = sum_l n_l / n."""
        return sum(l.n for l in self.levels) / self.levels[0].n


def _apply(Mx, X):
    return X if Mx is None else Mx @ X


def relax_homogeneous(lev: Level, U: np.ndarray, V: np.ndarray, p: Params):
    for _ in range(p.nu_setup):
        V = smoothing.jacobi(lev.B, lev.d, V, None, p.omega)
        Un = smoothing.jacobi(lev.Bt, lev.d, U, None, p.omega)
        Un[:, 0] = U[:, 0]
        U = Un
    return U, V


def rayleigh(lev: Level, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """eq. singular_value per column."""
    BV = lev.B @ V
    MU = _apply(lev.M, U)
    NV = _apply(lev.N, V)
    num = np.einsum("ik,ik->k", U, BV)
    den = np.sqrt(np.einsum("ik,ik->k", U, MU)) * np.sqrt(np.einsum("ik,ik->k", V, NV))
    return num / den


def relax_inhomogeneous(lev: Level, sig, U, V, p: Params):
    """Algorithm 1, second smoothing loop, with the sigma update."""
    for _ in range(p.nu_setup):
        rv = _apply(lev.M, U) * sig[None, :]
        ru = _apply(lev.N, V) * sig[None, :]
        Vn = smoothing.jacobi(lev.B, lev.d, V, rv, p.omega)
        Un = smoothing.jacobi(lev.Bt, lev.d, U, ru, p.omega)
        U, V = Un, Vn
        sig = rayleigh(lev, U, V)
    return sig, U, V


def split(lev: Level, l: int, p: Params):
    if p.coarsening == "geometric":
        nx, ny = lev.grid
        cf, cmap, cgrid = coarsening.geometric(nx, ny)
        J = coarsening.geometric_sets(nx, ny, cf)
        return cf, cmap, J, cgrid
    cf, cmap = coarsening.greedy_mis(lev.B, lev.Bt, p.seed, l)
    J = coarsening.graph_sets(lev.B, lev.Bt, cf, p.c_min, p.c_max)
    return cf, cmap, J, None


def make_level(B: sp.csr_matrix, M=None, N=None, grid=None) -> Level:
    return Level(n=B.shape[0], B=B, Bt=operators.transpose(B), d=operators.jacobi_divisor(B),
                 M=M, N=N, grid=grid)


def is_coarsest(lev: Level, l: int, p: Params) -> bool:
    if l + 1 >= p.max_levels or lev.n <= p.coarse_min:
        return True
    if p.coarsening == "geometric" and max(lev.grid) < 3:
        return True
    return False


def bamg_mle(H: Hierarchy, l: int, U: np.ndarray, V: np.ndarray, sig=None):
    """Algorithm 1 on level l; returns (sigma, U_l, V_l).  With sig given
    (a subsequent cycle) the first smoothing is the inhomogeneous one."""
    p = H.params
    lev = H.levels[l]
    if is_coarsest(lev, l, p):
        Bd = lev.B.toarray()
        Md = np.eye(lev.n) if lev.M is None else lev.M.toarray()
        Nd = np.eye(lev.n) if lev.N is None else lev.N.toarray()
        H.Bpinv = coarsest.pinv_drop_smallest(Bd)
        return coarsest.generalized_triplets(Bd, Md, Nd, p.r)
    if sig is None:
        U, V = relax_homogeneous(lev, U, V, p)
    else:
        sig, U, V = relax_inhomogeneous(lev, sig, U, V, p)
    r = V.shape[1]
    V = interp.normalise(V)
    U = interp.normalise(U, range(1, r))
    lev.s = interp.weights(lev.B, V)
    lev.t = interp.weights(lev.Bt, U, range(1, r))
    cf, cmap, J, cgrid = split(lev, l, p)
    lev.cf, lev.cmap, lev.J = cf, cmap, J
    lev.P = interp.ls_interpolation(V, lev.s, cf, cmap, J, p.ls_ridge)
    if p.restriction == "average":
        lev.Qt = interp.averaging_restriction_T(cf, cmap, J, lev.n)
    else:
        lev.Qt = interp.ls_restriction_T(U, lev.t, cf, cmap, J, p.ls_ridge)
    lev.Q = operators.transpose(lev.Qt)
    Bc = operators.galerkin(lev.Q, lev.B, lev.P)
    Mc = operators.spmatmul(lev.Q, lev.Qt if lev.M is None
                            else operators.spmatmul(lev.M, lev.Qt))
    Pt = operators.transpose(lev.P)
    Nc = operators.spmatmul(Pt, lev.P if lev.N is None
                            else operators.spmatmul(lev.N, lev.P))
    H.levels.append(make_level(Bc, Mc, Nc, cgrid))
    sig, Uc, Vc = bamg_mle(H, l + 1, U[cf], V[cf], sig)
    U = lev.Qt @ Uc
    V = lev.P @ Vc
    return relax_inhomogeneous(lev, sig, U, V, p)


def initial_x(sig: np.ndarray, V: np.ndarray) -> np.ndarray:
    """x^(0): the finest v with the smallest |sigma|, positive sum, unit 1-norm."""
    v = V[:, int(np.argmin(np.abs(sig)))].copy()
    if v.sum() < 0:
        v = -v
    return v / np.abs(v).sum()


def bamg_setup(A: sp.csr_matrix, p: Params, grid=None, U0=None, V0=None) -> Hierarchy:
    """Build B = I - A and run p.cycles bootstrap cycles (Algorithm 1)."""
    A = sp.csr_matrix(A)
    operators.validate_stochastic(A)
    B = operators.build_B(A)
    H = Hierarchy(params=p)
    H.levels.append(make_level(B, None, None, grid))
    if U0 is None or V0 is None:
        U0, V0 = rng.initial_test_vectors(p.seed, B.shape[0], p.r)
    sig, U, V = bamg_mle(H, 0, U0.copy(), V0.copy())
    for _ in range(1, p.cycles):
        del H.levels[1:]                       # rebuild below the finest level
        sig, U, V = bamg_mle(H, 0, U, V, sig)
    H.sigma, H.U, H.V = sig, U, V
    H.x0 = initial_x(sig, V)
    prepare_smoother(H)
    return H


def prepare_smoother(H: Hierarchy) -> None:
    """Row orders of the Gauss-Seidel V-cycle smoother on every non-coarsest
    level: the greedy colouring of the level's symmetrised graph (priorities
    SplitMix64 stream 6144 + l), rows by colour then index; or the natural
    order."""
    p = H.params
    for l, lev in enumerate(H.levels[:-1]):
        if p.smoother == "mcgs":
            lev.colour = smoothing.level_colouring(lev.B, lev.Bt, p.seed, l)
            lev.order = smoothing.multicolour_order(lev.colour)
        elif p.smoother == "gs":
            lev.order = np.arange(lev.n)
