"""The pair stream (abx_bvh_pairs): every unordered neighbour pair of a
hierarchy's points exactly once, as the paper's pair traversal hands them to
its callback F (subsection "Pair traversal").  The set must equal the
oracle's pair list exactly (integers: exact equality), also when delivered in
many small chunks, with pairs at exactly eps and at eps = 0."""
import numpy as np
import pytest

import oracle
from cases import _clumpy
from workloads import clumps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10743_gb300 import binding
    binding.lib()
    assert binding.device_status() == 0
    return binding


def sorted_rows(a):
    a = np.asarray(a, dtype=np.int64).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def lattice(side, spacing, keep, seed):
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    p = (g * spacing).astype(np.float32)
    p = p[rng.random(len(p)) < keep]
    return p[rng.permutation(len(p))]


CASES = [("clumpy", lambda: _clumpy(np.random.default_rng(21), 20_000, 12, 0.01), 0.01, 4),
         ("halo-mix", lambda: clumps(50_000, 60, 22, a0=0.01), 0.004, 8),
         ("lattice-at-eps", lambda: lattice(20, 2.0 ** -5, 0.7, 23), 2.0 ** -5, 2),
         ("duplicates-eps0", lambda: np.repeat(np.random.default_rng(24).random((2000, 3)).astype(np.float32),
                                               3, 0), 0.0, 1)]


@pytest.mark.parametrize("name,make,eps,leaf", CASES, ids=[c[0] for c in CASES])
def test_pairs_equal_oracle(abx, name, make, eps, leaf):
    p = make()
    h = abx.BVH(torch.from_numpy(p).cuda(), leaf_size=leaf)
    got = sorted_rows(h.pairs(eps).cpu().numpy())
    want = oracle.pairs(p, eps)
    assert abx.device_status() == 0
    assert got.shape == want.shape, (name, got.shape, want.shape)
    assert np.array_equal(got, want), name
    h.close()


def test_pairs_in_small_chunks(abx):
    p = _clumpy(np.random.default_rng(25), 8000, 8, 0.01)
    eps = 0.012
    h = abx.BVH(torch.from_numpy(p).cuda(), leaf_size=4)
    out = torch.empty((300, 2), dtype=torch.int32, device="cuda")
    cursor, parts, calls = 0, [], 0
    while cursor < len(p):
        rc, nxt, wrote = h.pairs_chunk(eps, cursor, out)
        assert rc == 0 and nxt > cursor and 0 <= wrote <= 300
        parts.append(out[:wrote].cpu().numpy().copy())
        cursor, calls = nxt, calls + 1
    assert calls > 3
    got = np.concatenate(parts)
    assert (got[:, 0] < got[:, 1]).all()
    assert np.array_equal(sorted_rows(got), oracle.pairs(p, eps))
    # the same order as one large call
    assert np.array_equal(got, h.pairs(eps, cap=1 << 20).cpu().numpy())
    h.close()


def test_pairs_buffer_too_small_for_one_point(abx):
    p = np.zeros((50, 3), np.float32)  # 50 identical points: the first has 49 pairs
    h = abx.BVH(torch.from_numpy(p).cuda())
    out = torch.empty((10, 2), dtype=torch.int32, device="cuda")
    rc, cur, wrote = h.pairs_chunk(0.0, 0, out)
    assert rc == abx.ABX_ENOMEM and cur == 0 and wrote == 0
    assert h.pairs(0.0, cap=10).shape[0] == 50 * 49 // 2
    h.close()


def test_pair_count_at_scale(abx):
    p = clumps(1 << 20, 1250, 26)
    eps = float(np.float32(0.168 / (1 << 20) ** (1 / 3)))
    h = abx.BVH(torch.from_numpy(p).cuda(), leaf_size=8)
    got = h.pairs(eps)
    assert got.shape[0] == oracle.pair_count(p, eps)
    g = got.cpu().numpy()
    # every pair really is a neighbour pair, and no pair repeats
    k = np.random.default_rng(0).choice(len(g), min(2000, len(g)), replace=False)
    assert all(oracle.pred(p[a], p[b], eps) for a, b in g[k])
    assert len(np.unique(g[:, 0].astype(np.int64) << 32 | g[:, 1])) == len(g)
    h.close()
