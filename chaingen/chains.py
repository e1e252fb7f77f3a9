"""Generators of irreducible Markov chains (Section 2 and Section 7 workloads).

Every generator returns a :class:`Chain` whose ``row_ptr/col/val`` hold the CSR
of the column-stochastic transition matrix ``A`` with ``a_ij = p_ji`` (row i
lists the probabilities of entering state i), column indices sorted ascending.

Workloads (Section 7):
  * ``uniform2d``    - uniform two-dimensional network (Table uniform2d):
                       from each state the walk moves to every lattice
                       neighbour with probability 1/(number of neighbours).
  * ``lattice2d``    - the same lattice with symmetric random edge weights
                       U(0.5, 1.5); probabilities are weight / weighted degree.
  * ``tandem``       - two queues in series (Table tandem): arrival, service
                       at station 1 (moves a customer to station 2) and service
                       at station 2, rates renormalised over the moves that
                       are feasible in each state.
  * ``birth_death``  - one-dimensional birth-death chain (Table birthdeath).
  * ``delaunay_walk``- random walk on the Delaunay triangulation of uniform
                       random points in the unit square (Table planargraph),
                       probability 1/degree to each neighbour.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Chain:
    """CSR of a column-stochastic ``A`` plus descriptive metadata."""
    name: str
    n: int
    row_ptr: np.ndarray          # int32[n+1]
    col: np.ndarray              # int32[nnz]
    val: np.ndarray              # float64[nnz]
    nx: int = 0                  # grid shape (0 = no grid)
    ny: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def kind(self) -> str:
        """Generator family: lattice, uniform, tandem, birthdeath, delaunay."""
        return self.name.rstrip("0123456789x")

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.row_ptr),
                             shape=(self.n, self.n))


def _from_moves(name, n, src, dst, prob, **kw) -> Chain:
    """Assemble A from a list of moves src -> dst with probability prob."""
    A = sp.csr_matrix((prob.astype(np.float64), (dst, src)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return Chain(name=name, n=n, row_ptr=A.indptr.astype(np.int32),
                 col=A.indices.astype(np.int32), val=A.data.astype(np.float64),
                 **kw)


def _lattice_edges(nx: int, ny: int):
    """Undirected 4-neighbour edges of an nx-by-ny grid, state s = i*ny + j."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(nx, ny)
    e1 = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    e2 = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    return np.concatenate([e1, e2], axis=0)


def lattice2d(nx: int, ny: int | None = None, seed: int = 1,
              wlo: float = 0.5, whi: float = 1.5) -> Chain:
    """Random walk on a weighted 5-point lattice with symmetric edge weights.

    Weights w_e ~ U(wlo, whi) from ``numpy.random.default_rng(seed)``; from
    state s the walk moves to neighbour t with probability w_st / W_s,
    W_s = sum_t w_st (the weighted degree, kept in ``meta['wdeg']``).
    """
    ny = nx if ny is None else ny
    n = nx * ny
    edges = _lattice_edges(nx, ny)
    rng = np.random.default_rng(seed)
    w = rng.uniform(wlo, whi, size=edges.shape[0])
    src = np.concatenate([edges[:, 0], edges[:, 1]])
    dst = np.concatenate([edges[:, 1], edges[:, 0]])
    ww = np.concatenate([w, w])
    wdeg = np.bincount(src, weights=ww, minlength=n)
    ch = _from_moves(f"lattice{nx}x{ny}", n, src, dst, ww / wdeg[src],
                     nx=nx, ny=ny)
    ch.meta["wdeg"] = wdeg
    return ch


def uniform2d(nx: int, ny: int | None = None) -> Chain:
    """Uniform two-dimensional network: probability 1/deg to each neighbour."""
    ny = nx if ny is None else ny
    n = nx * ny
    edges = _lattice_edges(nx, ny)
    src = np.concatenate([edges[:, 0], edges[:, 1]])
    dst = np.concatenate([edges[:, 1], edges[:, 0]])
    deg = np.bincount(src, minlength=n).astype(np.float64)
    ch = _from_moves(f"uniform{nx}x{ny}", n, src, dst, 1.0 / deg[src],
                     nx=nx, ny=ny)
    ch.meta["wdeg"] = deg
    return ch


def tandem(N: int, lam: float = 10 / 31, mu1: float = 11 / 31,
           mu2: float = 10 / 31) -> Chain:
    """Tandem queueing network with queue lengths 0..N-1 at both stations.

    State (i, j) = (customers at station 1, customers at station 2), index
    s = i*N + j.  Moves: arrival (i,j)->(i+1,j) [rate lam, i < N-1];
    service 1 (i,j)->(i-1,j+1) [rate mu1, i > 0 and j < N-1]; service 2
    (i,j)->(i,j-1) [rate mu2, j > 0].  Probabilities are the rates divided by
    the total rate of the moves feasible in that state (no self-loops).
    """
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    i = i.ravel(); j = j.ravel()
    s = i * N + j
    m_arr = i < N - 1
    m_s1 = (i > 0) & (j < N - 1)
    m_s2 = j > 0
    tot = lam * m_arr + mu1 * m_s1 + mu2 * m_s2
    src = np.concatenate([s[m_arr], s[m_s1], s[m_s2]])
    dst = np.concatenate([s[m_arr] + N, s[m_s1] - N + 1, s[m_s2] - 1])
    rate = np.concatenate([np.full(m_arr.sum(), lam), np.full(m_s1.sum(), mu1),
                           np.full(m_s2.sum(), mu2)])
    ch = _from_moves(f"tandem{N}x{N}", N * N, src, dst, rate / tot[src],
                     nx=N, ny=N)
    ch.meta.update(lam=lam, mu1=mu1, mu2=mu2)
    return ch


def birth_death(n: int, mu: float = 0.96) -> Chain:
    """Birth-death chain on states 0..n-1 (Table birthdeath, mu = 0.96).

    Interior states move right with probability 1/(1+mu) and left with
    probability mu/(1+mu); the end states move inwards with probability 1.
    """
    k = np.arange(n)
    up = np.where(k == 0, 1.0, 1.0 / (1.0 + mu))
    dn = np.where(k == n - 1, 1.0, mu / (1.0 + mu))
    m_up = k < n - 1
    m_dn = k > 0
    src = np.concatenate([k[m_up], k[m_dn]])
    dst = np.concatenate([k[m_up] + 1, k[m_dn] - 1])
    prob = np.concatenate([up[m_up], dn[m_dn]])
    ch = _from_moves(f"birthdeath{n}", n, src, dst, prob, nx=n, ny=1)
    ch.meta.update(mu=mu, p_up=up, p_dn=dn)
    return ch


def _delaunay_edges(pts: np.ndarray) -> np.ndarray:
    from scipy.spatial import Delaunay
    tri = Delaunay(pts).simplices.astype(np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [0, 2]]])
    e.sort(axis=1)
    n = pts.shape[0]
    key = np.unique(e[:, 0] * n + e[:, 1])
    return np.stack([key // n, key % n], axis=1)


def delaunay_walk(n: int, seed: int = 3, cache_dir: str | None = None) -> Chain:
    """Uniform random walk on the Delaunay graph of n uniform points.

    Points ~ U([0,1]^2) from ``numpy.random.default_rng(seed)``; the edges of
    the triangulation come from ``scipy.spatial.Delaunay``.  From each point
    the walk moves to every neighbour with probability 1/deg.  Large graphs
    may be cached as ``.npz`` under ``cache_dir``.
    """
    path = None
    if cache_dir:
        path = os.path.join(cache_dir, f"delaunay_{n}_{seed}.npz")
        if os.path.exists(path):
            z = np.load(path)
            ch = Chain(name=f"delaunay{n}", n=n, row_ptr=z["row_ptr"],
                       col=z["col"], val=z["val"])
            ch.meta["deg"] = z["deg"]
            return ch
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    edges = _delaunay_edges(pts)
    src = np.concatenate([edges[:, 0], edges[:, 1]])
    dst = np.concatenate([edges[:, 1], edges[:, 0]])
    deg = np.bincount(src, minlength=n).astype(np.float64)
    ch = _from_moves(f"delaunay{n}", n, src, dst, 1.0 / deg[src])
    ch.meta["deg"] = deg
    if path:
        os.makedirs(cache_dir, exist_ok=True)
        np.savez(path, row_ptr=ch.row_ptr, col=ch.col, val=ch.val, deg=deg)
    return ch


def chain_mix(count: int, seed: int = 4, side_lo: int = 32, side_hi: int = 256,
              del_lo: int = 1024, del_hi: int = 65536, log_sizes: bool = False) -> list:
    """Seeded mix of weighted lattices, tandem queues and Delaunay walks.
    Sizes are uniform in the side (lattices, queues) and in the point count
    (Delaunay walks), or with log_sizes uniform in their logarithms (about
    4.3M states for 256 chains instead of 7.4M)."""
    rng = np.random.default_rng(seed)

    def draw(lo, hi):
        if log_sizes:
            return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
        return int(rng.integers(lo, hi + 1))

    out = []
    for c in range(count):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            side = draw(side_lo, side_hi)
            out.append(lattice2d(side, side, seed=int(rng.integers(1 << 30))))
        elif kind == 1:
            side = draw(side_lo, side_hi)
            out.append(tandem(side))
        else:
            npts = draw(del_lo, del_hi)
            out.append(delaunay_walk(npts, seed=int(rng.integers(1 << 30))))
    return out


def to_dense(ch: Chain) -> np.ndarray:
    return ch.csr().toarray()


def training_mix(count: int = 512, seed: int = 6, lo: int = 64, hi: int = 512) -> list:
    """Seeded training chains of the interpolation network: tandem queues and
    weighted lattices alternating, sides uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(rng.integers(lo, hi + 1))
        out.append(tandem(side) if k % 2 == 0 else lattice2d(side, side, seed=int(rng.integers(1 << 30))))
    return out

