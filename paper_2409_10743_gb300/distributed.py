"""Domain decomposition: one point set spread over several processes (one GPU
each), clustered exactly as if it were one set.

The paper's HACC runs put one MPI rank on each GPU, every rank owning the
particles of a sub-volume plus an overload layer of copies from its
neighbours, and ArborX searches across ranks (sections "ArborX library" and
the HACC application).  Here every rank owns any subset of the points (slabs
of the box are the usual choice) and calls ``dbscan`` collectively:

1. the bounding boxes of all ranks' owned points are gathered;
2. ghosts: every rank sends every other rank its owned points that lie within
   eps of that rank's box, by the same rounded box test the traversals prune
   with (it never drops a neighbour), so every neighbour of an owned point is
   present locally;
3. core flags of the owned points: neighbour counts over the local set (owned
   + ghosts), capped at minPts (``abx_bvh_count``) -- exact, since every
   neighbour is local; the ghosts' core flags come back from their owners;
4. local clusters: components of the core-core neighbour pairs among the local
   points (``abx_bvh_pairs``), each keyed by its smallest global core index;
5. global merge: a core ghost lies in its owner's cluster and in the local one;
   rank 0 joins these equivalences from all ranks and every local key learns
   the global K, the smallest core index of its cluster;
6. borders (owned, not core, with a core neighbour) join the neighbouring
   cluster with the smallest K; a cluster's id is the smallest index over its
   core and border points, a global minimum per cluster.

Points are identified by global indices (``gid``); the returned labels are
global cluster ids (-1 noise), equal to what ``abx_dbscan`` returns for the
whole set.  The exchanges run over ``torch.distributed`` (gloo or any backend
with point-to-point sends) on host tensors; only the neighbour counts and the
pair stream run on the GPU, through the C ABI.  The per-rank work is
independent: no kernel waits on another rank.
"""
from __future__ import annotations

import numpy as np


class CudaEngine:
    """Local neighbour queries on this process's GPU through the C ABI."""

    def counts(self, local: np.ndarray, n_owned: int, eps: float, cap: int) -> np.ndarray:
        import torch

        from . import binding
        t = torch.from_numpy(np.ascontiguousarray(local, np.float32)).cuda()
        h = binding.BVH(t)
        try:
            c = h.count(t[:n_owned], eps, cap)
            torch.cuda.synchronize()
            return c.cpu().numpy().astype(np.int64)
        finally:
            h.close()

    def pairs(self, local: np.ndarray, eps: float) -> np.ndarray:
        import torch

        from . import binding
        t = torch.from_numpy(np.ascontiguousarray(local, np.float32)).cuda()
        h = binding.BVH(t)
        try:
            return h.pairs(eps).cpu().numpy().astype(np.int64)
        finally:
            h.close()


def box_reaches(p: np.ndarray, lo: np.ndarray, hi: np.ndarray, eps: float) -> np.ndarray:
    """Points whose rounded distance to the box [lo, hi] is at most eps: the
    per-axis gap max(0, lo - p, p - hi), squared and summed in FP32 in the
    neighbour test's order.  Rounding is monotone, so the value never exceeds
    the neighbour test's d2 to any point in the box."""
    p = np.asarray(p, np.float32)
    e2 = np.float32(eps) * np.float32(eps)
    d = np.maximum(np.float32(0), np.maximum(lo.astype(np.float32) - p, p - hi.astype(np.float32)))
    s = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    return (s + d[:, 2] * d[:, 2]) <= e2


def _exchange(dist, group, send: list, width: int, dtype) -> list:
    """Point-to-point all-to-all of variable-length 2-D arrays: send[q] goes
    to rank q; returns what every rank sent to this one."""
    import torch
    ws, me = dist.get_world_size(group), dist.get_rank(group)
    tdt = {np.float32: torch.float32, np.int64: torch.int64}[dtype]
    counts = [torch.tensor([len(send[q]) if q != me else 0], dtype=torch.int64) for q in range(ws)]
    rc = [torch.zeros(1, dtype=torch.int64) for _ in range(ws)]
    reqs = []
    for q in range(ws):
        if q != me:
            reqs.append(dist.isend(counts[q], q, group=group))
            reqs.append(dist.irecv(rc[q], q, group=group))
    for r in reqs:
        r.wait()
    out = [np.zeros((0, width), dtype) for _ in range(ws)]
    reqs, bufs = [], {}
    for q in range(ws):
        if q == me:
            continue
        if len(send[q]):
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(send[q], dtype).reshape(-1, width)),
                                   q, group=group))
        n = int(rc[q].item())
        if n:
            bufs[q] = torch.zeros((n, width), dtype=tdt)
            reqs.append(dist.irecv(bufs[q], q, group=group))
    for r in reqs:
        r.wait()
    for q, b in bufs.items():
        out[q] = b.numpy()
    return out


def _components(n: int, edges: np.ndarray) -> np.ndarray:
    """Connected component of each of n nodes over the edge list (k, 2)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    if len(edges) == 0:
        return np.arange(n)
    a = coo_matrix((np.ones(len(edges), np.int8), (edges[:, 0], edges[:, 1])), shape=(n, n))
    return connected_components(a, directed=False)[1]


def _lookup(table: dict, k: np.ndarray) -> np.ndarray:
    """table[k] where present, else k itself (vectorised)."""
    if not table or len(k) == 0:
        return k.copy()
    fk = np.fromiter(table.keys(), np.int64, len(table))
    fv = np.fromiter(table.values(), np.int64, len(table))
    o = np.argsort(fk)
    fk, fv = fk[o], fv[o]
    i = np.minimum(np.searchsorted(fk, k), len(fk) - 1)
    return np.where(fk[i] == k, fv[i], k)


def dbscan(points: np.ndarray, gid: np.ndarray, eps: float, minpts: int, group=None, engine=None) -> np.ndarray:
    """Collective: every rank passes its owned points (float32 (n, 3)) and
    their global indices (int64 (n,)); returns their labels (int64 (n,)):
    the smallest global index of the point's cluster, -1 for noise."""
    import torch
    import torch.distributed as dist
    engine = engine or CudaEngine()
    ws, me = dist.get_world_size(group), dist.get_rank(group)
    pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    gid = np.ascontiguousarray(gid, np.int64).reshape(-1)
    n = len(pts)
    eps = float(np.float32(eps))

    # 1. every rank's box (an empty rank's box reaches nothing)
    box = np.full(6, np.nan, np.float32)
    if n:
        box = np.concatenate([pts.min(0), pts.max(0)]).astype(np.float32)
    boxes = [torch.zeros(6) for _ in range(ws)]
    dist.all_gather(boxes, torch.from_numpy(box), group=group)
    boxes = [b.numpy() for b in boxes]

    # 2. ghosts: the owned points within eps of each other rank's box
    sent_idx = [np.zeros(0, np.int64) for _ in range(ws)]
    for q in range(ws):
        if q != me and n and not np.isnan(boxes[q][0]):
            sent_idx[q] = np.nonzero(box_reaches(pts, boxes[q][:3], boxes[q][3:], eps))[0]
    send = [np.concatenate([pts[s].view(np.int32).astype(np.int64), gid[s, None]], 1) for s in sent_idx]
    got = _exchange(dist, group, send, 4, np.int64)
    ghost = np.concatenate(got) if any(len(g) for g in got) else np.zeros((0, 4), np.int64)
    gpts = ghost[:, :3].astype(np.int32).view(np.float32)
    ggid = ghost[:, 3]
    local = np.concatenate([pts, gpts]) if len(gpts) else pts
    lgid = np.concatenate([gid, ggid])
    m = len(local)

    # 3. core flags: owned ones counted here, ghosts' from their owners
    core = np.zeros(m, bool)
    if n:
        core[:n] = engine.counts(local, n, eps, minpts) >= minpts
    back = _exchange(dist, group, [core[s].astype(np.int64)[:, None] for s in sent_idx], 1, np.int64)
    core[n:] = np.concatenate([b[:, 0] for b in back]).astype(bool) if len(gpts) else core[n:]

    # 4. local clusters of core points, keyed by their smallest global index
    pairs = engine.pairs(local, eps) if m > 1 else np.zeros((0, 2), np.int64)
    cc = pairs[core[pairs[:, 0]] & core[pairs[:, 1]]] if len(pairs) else pairs
    comp = _components(m, cc)
    key = np.full(m, np.iinfo(np.int64).max, np.int64)
    kc = np.full(comp.max() + 1 if m else 0, np.iinfo(np.int64).max, np.int64)
    np.minimum.at(kc, comp[core], lgid[core])
    key[core] = kc[comp[core]]

    # 5. global merge: (global index, local key) of every core point that is
    #    somebody's ghost (here) or sent as one (the owner's side)
    boundary = np.zeros(m, bool)
    boundary[n:] = True
    for s in sent_idx:
        boundary[s] = True
    sel = boundary & core
    mine = np.stack([lgid[sel], key[sel]], 1)
    allp = [None] * ws if me == 0 else None
    dist.gather_object(mine, allp, dst=0, group=group)
    final_of = [None]
    if me == 0:
        e = np.concatenate(allp) if allp else np.zeros((0, 2), np.int64)
        ids, inv = np.unique(e.reshape(-1), return_inverse=True)
        cls = _components(len(ids), inv.reshape(-1, 2))
        keys = np.unique(e[:, 1])
        is_key = np.isin(ids, keys)
        best = np.full(cls.max() + 1 if len(ids) else 0, np.iinfo(np.int64).max, np.int64)
        np.minimum.at(best, cls[is_key], ids[is_key])
        final_of = [dict(zip(ids[is_key].tolist(), best[cls[is_key]].tolist()))]
    dist.broadcast_object_list(final_of, src=0, group=group)
    final = final_of[0]
    K = np.full(m, -1, np.int64)
    K[core] = _lookup(final, key[core])

    # 6. borders: owned non-core points take the smallest K among core neighbours
    border_k = np.full(n, np.iinfo(np.int64).max, np.int64)
    if len(pairs):
        for a, b in ((0, 1), (1, 0)):
            i, j = pairs[:, a], pairs[:, b]
            take = (i < n) & ~core[i] & core[j]
            np.minimum.at(border_k, i[take], K[j[take]])
    is_border = (border_k != np.iinfo(np.int64).max) & ~core[:n]
    bk, bg = border_k[is_border], gid[is_border]
    bmin = {}
    if len(bk):
        order = np.lexsort((bg, bk))
        first = np.r_[True, bk[order][1:] != bk[order][:-1]]
        bmin = dict(zip(bk[order][first].tolist(), bg[order][first].tolist()))
    allb = [None] * ws if me == 0 else None
    dist.gather_object(bmin, allb, dst=0, group=group)
    merged = [None]
    if me == 0:
        out = {}
        for d in allb:
            for k, v in d.items():
                out[k] = min(out.get(k, v), v)
        merged = [out]
    dist.broadcast_object_list(merged, src=0, group=group)
    bmin = merged[0]

    labels = np.full(n, -1, np.int64)
    owned_core = core[:n]
    kc_own = K[:n][owned_core]
    labels[owned_core] = np.minimum(kc_own, _lookup(bmin, kc_own))
    labels[is_border] = np.minimum(bk, _lookup(bmin, bk))
    return labels
