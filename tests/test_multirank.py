"""The N > 1 benchmark path on CPU: two gloo ranks (127.0.0.1).  Each rank
clusters its own replica (distinct seeds, no data-path collective) and the
reported time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    from workloads import CONFIGS
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.reduce_max(10.0 + 5 * rank, ws)
    cfg = bench.rank_config(CONFIGS["fof-clumps-134M"], rank, ws)
    dist.barrier()
    out.put((rank, t, cfg.seed, cfg.n, cfg.eps))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_distinct_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]          # both see the slowest rank
    assert res[0][2] != res[1][2]                        # independent replicas
    assert res[0][3] == res[1][3] and res[0][4] == res[1][4]  # same workload shape


def test_single_rank_is_identity():
    import bench
    from workloads import CONFIGS
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.rank_config(CONFIGS["fof-clumps-134M"], 0, 1) is CONFIGS["fof-clumps-134M"]
