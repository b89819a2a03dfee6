"""Brute-force DBSCAN straight from the definitions, used to pin the oracle.

O(n^2) and independent of the oracle's code: a dense adjacency test in numpy
float32 (every elementwise operation rounds on its own; numpy never fuses a
multiply and an add) and breadth-first search over the core points, instead of
the oracle's grid and union-find.  Definitions: paper, subsection "DBSCAN
algorithm" (eps-neighbourhood including the point itself, core iff
|N_eps| >= minPts, border = non-core reachable from a core point, noise = the
rest).  The border tie rule and the cluster id are the library's readings:
a border point joins the neighbouring cluster whose smallest core index is
smallest, and a cluster's id is its smallest member index.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency_rows(p: np.ndarray, eps: float, rows: slice) -> np.ndarray:
    """Boolean block A[i, j] = pred(i, j) for i in rows, all j."""
    p = np.asarray(p, dtype=np.float32)
    e2 = np.float32(eps) * np.float32(eps)
    q = p[rows]
    dx = q[:, None, 0] - p[None, :, 0]
    dy = q[:, None, 1] - p[None, :, 1]
    dz = q[:, None, 2] - p[None, :, 2]
    xx = dx * dx
    yy = dy * dy
    zz = dz * dz
    s = xx + yy
    d2 = s + zz
    assert d2.dtype == np.float32
    return d2 <= e2


def neighbour_lists(p: np.ndarray, eps: float, block: int = 1024) -> list[np.ndarray]:
    n = len(p)
    out = []
    for s in range(0, n, block):
        a = adjacency_rows(p, eps, slice(s, min(n, s + block)))
        out.extend(np.nonzero(row)[0] for row in a)
    return out


def dbscan(p: np.ndarray, eps: float, minpts: int) -> np.ndarray:
    p = np.asarray(p, dtype=np.float32)
    n = len(p)
    nb = neighbour_lists(p, eps)
    core = np.array([len(x) >= minpts for x in nb], dtype=bool)
    comp = np.full(n, -1, dtype=np.int64)
    key = []  # smallest core index per component
    for s in range(n):
        if not core[s] or comp[s] >= 0:
            continue
        c = len(key)
        comp[s] = c
        members = [s]
        dq = deque([s])
        while dq:
            x = dq.popleft()
            for y in nb[x]:
                if core[y] and comp[y] < 0:
                    comp[y] = c
                    members.append(int(y))
                    dq.append(y)
        key.append(min(members))
    labels = np.full(n, -1, dtype=np.int64)
    cid = list(key)
    border_of = np.full(n, -1, dtype=np.int64)
    for b in range(n):
        if core[b]:
            continue
        cs = [comp[y] for y in nb[b] if core[y]]
        if cs:
            border_of[b] = min(cs, key=lambda c: key[c])
            cid[border_of[b]] = min(cid[border_of[b]], b)
    for i in range(n):
        if core[i]:
            labels[i] = cid[comp[i]]
        elif border_of[i] >= 0:
            labels[i] = cid[border_of[i]]
    return labels.astype(np.int32)


def core_flags(p: np.ndarray, eps: float, minpts: int) -> np.ndarray:
    return np.array([len(x) >= minpts for x in neighbour_lists(p, eps)], dtype=bool)


def pair_count(p: np.ndarray, eps: float, block: int = 1024) -> int:
    n = len(p)
    total = 0
    for s in range(0, n, block):
        a = adjacency_rows(p, eps, slice(s, min(n, s + block)))
        total += int(a.sum()) - a.shape[0]  # drop the diagonal
    return total // 2


def fof_components(p: np.ndarray, eps: float, block: int = 2048) -> np.ndarray:
    """FoF labels as connected components of the eps-graph (scipy), isolated
    points as noise.  The minPts = 2 invariant of the paper's "Initial DBSCAN
    implementation" subsection."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    p = np.asarray(p, dtype=np.float32)
    n = len(p)
    rows, cols = [], []
    for s in range(0, n, block):
        a = adjacency_rows(p, eps, slice(s, min(n, s + block)))
        i, j = np.nonzero(a)
        rows.append(i + s)
        cols.append(j)
    i = np.concatenate(rows)
    j = np.concatenate(cols)
    g = sp.coo_matrix((np.ones(i.size, dtype=np.int8), (i, j)), shape=(n, n)).tocsr()
    _, comp = connected_components(g, directed=False)
    deg = np.bincount(i, minlength=n)  # includes the self-loop
    first = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(n))
    lab = first[comp]
    lab[deg < 2] = -1
    return lab.astype(np.int32)


def pair_histogram(p: np.ndarray, r_edges, block: int = 1024) -> np.ndarray:
    """Unordered pairs {i, j}, i != j, with fl(r_b^2) < d2 <= fl(r_{b+1}^2)."""
    p = np.asarray(p, dtype=np.float32)
    e = np.asarray(r_edges, dtype=np.float32)
    e2 = e * e
    n = len(p)
    hist = np.zeros(len(e) - 1, np.int64)
    for s in range(0, n, block):
        q = p[s:s + block]
        dx = q[:, None, 0] - p[None, :, 0]
        dy = q[:, None, 1] - p[None, :, 1]
        dz = q[:, None, 2] - p[None, :, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        i = np.arange(s, s + len(q))[:, None]
        j = np.arange(n)[None, :]
        d = d2[j > i]
        for b in range(len(e) - 1):
            hist[b] += int(((d > e2[b]) & (d <= e2[b + 1])).sum())
    return hist
