"""C/F splitting and interpolation sets J_i.

Geometric coarsening (Section 7, uniform 2D / tandem tables): the coarse
variables are every other grid point in both directions, i.e. the points
(i, j) with i and j even; J_i is the set of coarse points inside the 3x3 box
around a fine point (at most c = 4 of them).

Unstructured graphs (Section 7, planar graph table) use compatible relaxation
in the paper, which it does not spell out.  In its place this oracle uses the
greedy maximal independent set in a fixed priority order on the symmetrised
graph of B, and picks J_i among coarse neighbours by connection strength.

Coarse variables are numbered in ascending order of their fine index.
"""
import numpy as np
import scipy.sparse as sp

from . import rng

MIS_STREAM = 4096


def geometric(nx: int, ny: int):
    """C = {(i, j): i even and j even} on an nx-by-ny grid (s = i*ny + j)."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    cf = ((i % 2 == 0) & (j % 2 == 0)).ravel()
    cmap = np.full(nx * ny, -1, dtype=np.int64)
    cmap[cf] = np.arange(int(cf.sum()))
    return cf, cmap, ((nx + 1) // 2, (ny + 1) // 2)


def geometric_sets(nx: int, ny: int, cf: np.ndarray):
    """J_i for every fine point: coarse points of the 3x3 box, ascending."""
    J = {}
    for s in np.flatnonzero(~cf):
        i, j = divmod(int(s), ny)
        sel = []
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                a, b = i + di, j + dj
                if 0 <= a < nx and 0 <= b < ny and cf[a * ny + b]:
                    sel.append(a * ny + b)
        J[int(s)] = sorted(sel)
    return J


def symmetric_neighbours(B: sp.csr_matrix, Bt: sp.csr_matrix, i: int):
    """Off-diagonal neighbours of i in the graph of B + B^T with strengths.

    strength s_ij = |b_ij| + |b_ji| (a missing entry counts as 0).
    """
    out = {}
    for p in range(B.indptr[i], B.indptr[i + 1]):
        j = int(B.indices[p])
        if j != i:
            out[j] = out.get(j, 0.0) + abs(B.data[p])
    for p in range(Bt.indptr[i], Bt.indptr[i + 1]):
        j = int(Bt.indices[p])
        if j != i:
            out[j] = out.get(j, 0.0) + abs(Bt.data[p])
    return out


def mis_priorities(n: int, seed: int, level: int) -> np.ndarray:
    return rng.draw(seed, MIS_STREAM + level, n)


def mis_order(key: np.ndarray) -> np.ndarray:
    """Vertices by decreasing priority, equal priorities by increasing index."""
    n = key.shape[0]
    return np.lexsort((np.arange(n), ~key))


def greedy_mis(B: sp.csr_matrix, Bt: sp.csr_matrix, seed: int, level: int):
    """Greedy maximal independent set, vertices visited by priority.

    A vertex becomes coarse when no neighbour visited before it is coarse.
    """
    n = B.shape[0]
    key = mis_priorities(n, seed, level)
    Bs = (abs(B) + abs(Bt)).tocsr()
    cf = np.zeros(n, dtype=bool)
    blocked = np.zeros(n, dtype=bool)
    for v in mis_order(key):
        if blocked[v]:
            continue
        cf[v] = True
        nb = Bs.indices[Bs.indptr[v]:Bs.indptr[v + 1]]
        blocked[nb] = True
    cmap = np.full(n, -1, dtype=np.int64)
    cmap[cf] = np.arange(int(cf.sum()))
    return cf, cmap


def graph_sets(B: sp.csr_matrix, Bt: sp.csr_matrix, cf: np.ndarray,
               c_min: int, c_max: int):
    """J_i on a graph: strongest coarse neighbours, topped up from distance 2.

    Distance-1 coarse neighbours are ranked by strength (descending, ties by
    index) and the first c_max kept.  If fewer than c_min remain, coarse
    points two steps away are added, ranked by the largest product of
    strengths over the connecting points, until c_min are chosen.
    """
    J = {}
    for i in np.flatnonzero(~cf):
        i = int(i)
        nb = symmetric_neighbours(B, Bt, i)
        d1 = sorted(((-s, j) for j, s in nb.items() if cf[j]))
        sel = [j for _, j in d1[:c_max]]
        if len(sel) < c_min:
            cand = {}
            for k, sik in nb.items():
                for j, skj in symmetric_neighbours(B, Bt, k).items():
                    if j == i or not cf[j] or j in sel:
                        continue
                    w = sik * skj
                    if w > cand.get(j, -1.0):
                        cand[j] = w
            d2 = sorted(((-w, j) for j, w in cand.items()))
            sel += [j for _, j in d2[:c_min - len(sel)]]
        J[i] = sorted(sel)
    return J
