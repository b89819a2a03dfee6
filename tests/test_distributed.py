"""Domain decomposition (paper: one rank per GPU, each owning a sub-volume with
ghost copies from its neighbours): ranks owning parts of one point set, run as
gloo processes, must return together exactly the labels of the whole set
(the oracle's), for slab and scattered partitions, FoF and general minPts.

On CPU the ranks' local neighbour queries come from a brute-force engine (a
test stand-in for the GPU); the GPU test runs two processes that share the GPU,
each with the library's engine, exchanging over gloo (their kernels never wait
on each other)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class BruteEngine:
    """O(m^2) neighbour queries in numpy float32 (the neighbour test's op order)."""

    def counts(self, local, n_owned, eps, cap):
        import brute
        a = brute.adjacency_rows(local, eps, slice(0, n_owned))
        return np.minimum(a.sum(1), cap)

    def pairs(self, local, eps):
        import brute
        out = []
        for s in range(0, len(local), 512):
            a = brute.adjacency_rows(local, eps, slice(s, min(len(local), s + 512)))
            i, j = np.nonzero(a)
            i = i + s
            keep = j > i
            out.append(np.stack([i[keep], j[keep]], 1))
        return np.concatenate(out).astype(np.int64) if out else np.zeros((0, 2), np.int64)


def make_points(seed):
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, here)
    from cases import _clumpy
    return _clumpy(np.random.default_rng(seed), 3000, 10, 0.015)


def partition(p, ws, how, seed):
    if how == "slabs":
        edges = np.quantile(p[:, 0], np.linspace(0, 1, ws + 1))
        own = np.clip(np.searchsorted(edges, p[:, 0], side="right") - 1, 0, ws - 1)
    else:
        own = np.random.default_rng(seed).integers(0, ws, len(p))
    return own


def _worker(rank, ws, port, cfg, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as dist
    from paper_2409_10743_gb300 import distributed
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        p = make_points(cfg["seed"])
        own = partition(p, ws, cfg["how"], cfg["seed"])
        gid = np.nonzero(own == rank)[0]
        engine = BruteEngine() if cfg["engine"] == "brute" else None
        if engine is None:
            import torch as _t
            _t.cuda.set_device(0)
        lab = distributed.dbscan(p[gid], gid, cfg["eps"], cfg["minpts"], engine=engine)
        q.put((rank, gid, lab))
    finally:
        dist.destroy_process_group()


def run_ranks(ws, cfg):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, cfg, q)) for r in range(ws)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = make_points(cfg["seed"])
    lab = np.full(len(p), -2, np.int64)
    for _, gid, l in res:
        lab[gid] = l
    assert (lab != -2).all()
    return p, lab


@pytest.mark.parametrize("ws,how,minpts", [(2, "slabs", 2), (2, "slabs", 5), (3, "scattered", 4),
                                           (3, "slabs", 1)])
def test_ranks_equal_whole_set(ws, how, minpts):
    import oracle
    cfg = dict(seed=40 + ws + minpts, how=how, eps=0.02, minpts=minpts, engine="brute")
    p, lab = run_ranks(ws, cfg)
    assert np.array_equal(lab, oracle.dbscan(p, cfg["eps"], minpts))


def test_box_reach_is_conservative():
    """A point that passes the neighbour test with some point of a box always
    passes the rounded box test (no ghost is ever missed)."""
    import oracle
    from paper_2409_10743_gb300.distributed import box_reaches
    rng = np.random.default_rng(3)
    for _ in range(20):
        box = rng.random((40, 3)).astype(np.float32) * 0.1 + rng.random(3).astype(np.float32)
        lo, hi = box.min(0), box.max(0)
        q = (rng.random((400, 3)) * 0.3 + lo - 0.1).astype(np.float32)
        eps = 0.03
        near = np.array([any(oracle.pred(x, b, eps) for b in box) for x in q])
        assert not (near & ~box_reaches(q, lo, hi, eps)).any()


@pytest.mark.gpu
def test_two_processes_on_the_gpu():
    import oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = dict(seed=77, how="slabs", eps=0.02, minpts=5, engine="cuda")
    p, lab = run_ranks(2, cfg)
    assert np.array_equal(lab, oracle.dbscan(p, cfg["eps"], cfg["minpts"]))
    cfg = dict(seed=78, how="scattered", eps=0.02, minpts=2, engine="cuda")
    p, lab = run_ranks(2, cfg)
    assert np.array_equal(lab, oracle.dbscan(p, cfg["eps"], cfg["minpts"]))
