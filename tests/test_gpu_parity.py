"""GPU parity: labels from the CUDA library (through the C ABI) must equal the
oracle's bit for bit -- labels are integers, so the bar is exact equality --
on the hand cases, small seeded cases over many tuning parameters, and the
full-size configurations.  Also edge cases, determinism, and the device
status word."""
import numpy as np
import pytest

import oracle
from cases import _cases, _clumpy
from conftest import golden_cases
from workloads import CONFIGS, clumps, scaled

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


def gpu_labels(abx, p, eps, minpts, params=None):
    t = torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
    lab = abx.dbscan(t, eps, minpts, params=params)
    torch.cuda.synchronize()
    assert abx.device_status() == 0
    return lab.cpu().numpy()


def assert_same(got, want, what=""):
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{what}: {bad.size} of {got.size} labels differ; first at {bad[:8]}: "
                             f"got {got[bad[:8]]}, want {want[bad[:8]]}")


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_golden(abx, case):
    name, p, eps, minpts, want = case
    assert_same(gpu_labels(abx, p, eps, minpts), want, name)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_small_cases(abx, case):
    name, p, eps, minpts = case
    assert_same(gpu_labels(abx, p, eps, minpts), oracle.dbscan(p, eps, minpts), name)


PARAMS = [dict(leaf_size=1), dict(leaf_size=2), dict(leaf_size=8), dict(leaf_size=32),
          dict(dense_cells=-1), dict(sub_bits=3), dict(sub_bits=8), dict(block=128),
          dict(block=1024), dict(leaf_size=1, dense_cells=-1)]


@pytest.mark.parametrize("kw", PARAMS, ids=lambda k: ",".join(f"{a}={b}" for a, b in k.items()))
def test_parameters_never_change_labels(abx, kw):
    rng = np.random.default_rng(77)
    for minpts, eps, p in [(2, 0.02, _clumpy(rng, 6000, 12, 0.01)), (5, 0.03, _clumpy(rng, 6000, 12, 0.01)),
                           (2, 0.0, np.repeat(_clumpy(rng, 500, 5, 0.01), 3, axis=0))]:
        assert_same(gpu_labels(abx, p, eps, minpts, abx.Params(**kw)), oracle.dbscan(p, eps, minpts), str(kw))


def test_empty_and_single(abx):
    t = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    assert abx.dbscan(t, 0.1, 2).numel() == 0
    one = np.array([[0.5, 0.5, 0.5]], np.float32)
    assert gpu_labels(abx, one, 0.1, 1).tolist() == [0]
    assert gpu_labels(abx, one, 0.1, 2).tolist() == [-1]


def test_all_identical_points(abx):
    p = np.full((5000, 3), 0.25, np.float32)
    assert (gpu_labels(abx, p, 0.0, 2) == 0).all()
    assert (gpu_labels(abx, p, 0.0, 5001) == -1).all()
    assert (gpu_labels(abx, p, 0.1, 7) == 0).all()


def test_ragged_tiles(abx):
    """Sizes around the sort and scan tile (4096) and the block size."""
    rng = np.random.default_rng(3)
    for n in [255, 256, 257, 4095, 4096, 4097, 8193, 12289]:
        p = _clumpy(rng, n, 6, 0.01)
        for minpts in (2, 4):
            assert_same(gpu_labels(abx, p, 0.02, minpts), oracle.dbscan(p, 0.02, minpts), f"n={n}")


def test_unaligned_points(abx):
    """A points pointer that is not 16-byte aligned takes the scalar bounds path."""
    rng = np.random.default_rng(8)
    p = _clumpy(rng, 3001, 6, 0.01)
    flat = torch.from_numpy(np.concatenate([[0.0], p.ravel()]).astype(np.float32)).cuda()
    view = flat[1:].view(-1, 3)
    assert view.data_ptr() % 16 != 0
    lab = abx.dbscan(view, 0.02, 3)
    torch.cuda.synchronize()
    assert_same(lab.cpu().numpy(), oracle.dbscan(p, 0.02, 3), "unaligned")


def test_extreme_coordinates(abx):
    rng = np.random.default_rng(12)
    p = (_clumpy(rng, 4000, 6, 0.01) * 1e6 - 3e5).astype(np.float32)
    assert_same(gpu_labels(abx, p, 2e4, 3), oracle.dbscan(p, 2e4, 3), "scaled")
    p = (_clumpy(rng, 4000, 6, 0.01) * 1e-20).astype(np.float32)
    assert_same(gpu_labels(abx, p, 2e-22, 2), oracle.dbscan(p, 2e-22, 2), "tiny")
    # eps far larger than the extent: one cluster
    q = _clumpy(rng, 3000, 6, 0.01)
    assert_same(gpu_labels(abx, q, 10.0, 5), oracle.dbscan(q, 10.0, 5), "huge eps")


def test_deterministic(abx):
    p = clumps(200_000, 200, 31, a0=0.02)
    eps = 0.004
    a = gpu_labels(abx, p, eps, 2)
    for _ in range(3):
        assert np.array_equal(gpu_labels(abx, p, eps, 2), a)


def test_nonfinite_sets_status(abx):
    p = _clumpy(np.random.default_rng(2), 1000, 4, 0.01)
    p[17, 1] = np.nan
    t = torch.from_numpy(p).cuda()
    abx.dbscan(t, 0.02, 2)
    assert abx.device_status() == abx.ABX_ENONFINITE
    assert abx.device_status() == 0  # cleared


def test_host_entry_point(abx):
    p = clumps(100_000, 100, 41, a0=0.02)
    eps = 0.005
    assert_same(abx.dbscan_host(p, eps, 3), oracle.dbscan(p, eps, 3), "host")


def test_batch_equals_single(abx):
    rng = np.random.default_rng(5)
    sizes = [0, 1, 700, 5000, 33, 20000]
    segs = [_clumpy(rng, n, 5, 0.01) if n else np.zeros((0, 3), np.float32) for n in sizes]
    eps = [0.02, 0.1, 0.03, 0.02, 0.5, 0.01]
    mp = [2, 1, 5, 2, 3, 10]
    off = np.concatenate([[0], np.cumsum(sizes)])
    allp = torch.from_numpy(np.concatenate(segs).astype(np.float32)).cuda()
    lab = abx.dbscan_batch(allp, off, eps, mp)
    torch.cuda.synchronize()
    assert abx.device_status() == 0
    lab = lab.cpu().numpy()
    for k in range(len(sizes)):
        assert_same(lab[off[k]:off[k + 1]], oracle.dbscan(segs[k], eps[k], mp[k]), f"segment {k}")


def test_bvh_count_early_termination(abx):
    rng = np.random.default_rng(9)
    p = _clumpy(rng, 20000, 10, 0.02)
    q = _clumpy(rng, 3000, 10, 0.02)
    eps = 0.02
    import brute
    full = np.array([brute.adjacency_rows(np.concatenate([q[i:i + 1], p]), eps, slice(0, 1))[0, 1:].sum()
                     for i in range(200)])
    h = abx.BVH(torch.from_numpy(p).cuda(), leaf_size=4)
    info = h.info()
    assert info["n_points"] == len(p) and 1 <= info["n_leaves"] <= len(p) and info["levels"] >= 2
    for cap in (1, 5, 1000000):
        got = h.count(torch.from_numpy(q[:200]).cuda(), eps, cap).cpu().numpy()
        assert np.array_equal(got, np.minimum(full, cap))
    h.close()


@pytest.mark.parametrize("leaf_size", [1, 4, 8])
def test_bvh_first_hit(abx, leaf_size):
    """A first hit is some tree point within eps of the query (several can be
    right: check that the one returned is), and -1 exactly where no tree point
    is within eps (brute force)."""
    import brute
    rng = np.random.default_rng(19 + leaf_size)
    p = _clumpy(rng, 20000, 10, 0.02)
    q = np.concatenate([_clumpy(rng, 2000, 10, 0.02), rng.random((500, 3), dtype=np.float32) * 1.2 - 0.1])
    q = q.astype(np.float32)
    h = abx.BVH(torch.from_numpy(p).cuda(), leaf_size=leaf_size)
    for eps in (0.0, 0.004, 0.02):
        got = h.first_hit(torch.from_numpy(q).cuda(), eps).cpu().numpy()
        torch.cuda.synchronize()
        assert abx.device_status() == 0
        has = np.array([brute.adjacency_rows(np.concatenate([q[i:i + 1], p]), eps, slice(0, 1))[0, 1:].any()
                        for i in range(len(q))])
        assert np.array_equal(got >= 0, has), f"eps={eps}"
        for i in np.nonzero(got >= 0)[0]:
            assert 0 <= got[i] < len(p) and oracle.pred(q[i], p[got[i]], eps), (i, got[i])
    # points of the tree itself always hit (eps = 0: an exact duplicate, themselves)
    got = h.first_hit(torch.from_numpy(p[:300]).cuda(), 0.0).cpu().numpy()
    assert np.all(got >= 0) and np.all(np.all(p[got] == p[:300], axis=1))
    h.close()


# ---- full-size configurations ------------------------------------------------------

def _full(abx, name):
    cfg = CONFIGS[name]
    p = cfg.points()
    got = gpu_labels(abx, p, cfg.eps, cfg.minpts)
    want = oracle.dbscan(p, cfg.eps, cfg.minpts)
    assert_same(got, want, cfg.describe())
    return got


def test_full_fof_uniform_32k(abx):
    _full(abx, "fof-uniform-32K")


@pytest.mark.slow
def test_full_fof_clumps_16m(abx):
    _full(abx, "fof-clumps-16M")


@pytest.mark.slow
def test_full_fof_halos_16m(abx):
    _full(abx, "fof-halos-16M")


@pytest.mark.slow
def test_full_dbscan_blobs_10m(abx):
    _full(abx, "dbscan-blobs-10M")


@pytest.mark.slow
def test_full_fof_clumps_134m(abx):
    """2^27 points, FoF: the benchmark's workload, compared label by label with
    the library defaults and with the parameters the benchmark runs (the
    autotuner's pick on this workload: leaf 8, dense cells off, block 128)."""
    got = _full(abx, "fof-clumps-134M")
    cfg = CONFIGS["fof-clumps-134M"]
    bench = gpu_labels(abx, cfg.points(), cfg.eps, cfg.minpts,
                       abx.Params(leaf_size=8, dense_cells=-1, block=128))
    assert_same(bench, got, "benchmark parameters")


@pytest.mark.parametrize("name", ["fof-clumps-16M", "dbscan-blobs-10M", "fof-halos-16M"])
def test_scaled_configs(abx, name):
    cfg = scaled(CONFIGS[name], 300_000)
    p = cfg.points()
    assert_same(gpu_labels(abx, p, cfg.eps, cfg.minpts), oracle.dbscan(p, cfg.eps, cfg.minpts), cfg.describe())


def test_profile_api(abx):
    """Stage timers, counters and the launch counter on the default stream."""
    p = clumps(300_000, 300, 51, a0=0.02)
    t = torch.from_numpy(p).cuda()
    abx.profile_enable(True)
    try:
        n0 = abx.launch_count()
        abx.dbscan(t, 0.004, 2)
        ms = abx.profile_read()
        c = abx.profile_counters()
        n1 = abx.launch_count()
        abx.dbscan(t, 0.004, 5)
        ms5 = abx.profile_read()
    finally:
        abx.profile_enable(False)
    assert set(ms) >= {"bounds", "sort", "union", "finalize"}
    assert all(v >= 0 for v in ms.values()) and ms["union"] > 0 and ms["count"] == 0
    assert ms5["count"] > 0 and ms5["border"] > 0
    assert 1 <= c["radix_passes"] <= 8 and 1 <= c["leaves"] <= len(p) and c["morton_bits"] <= 21
    assert n1 - n0 >= 15


@pytest.mark.parametrize("minpts", [2, 4])
@pytest.mark.parametrize("kw", [dict(dense_cells=-1, leaf_size=2), dict(leaf_size=4), dict(dense_cells=-1, leaf_size=1)],
                         ids=["leaf2", "dense-leaf4", "leaf1"])
def test_candidate_list_overflow(abx, kw, minpts):
    """Leaves with more candidate leaves than the per-leaf list holds fall back
    to the rope walk from where the list ran out (the traversal counters then
    show node visits); leaves with few candidates visit no node at all.  Both
    must give the oracle's labels."""
    p = clumps(60_000, 40, 71 + minpts, a0=0.03)
    t = torch.from_numpy(p).cuda()
    for eps, overflow in [(0.02, True), (0.0005, False)]:
        abx.profile_enable(2)
        try:
            lab = abx.dbscan(t, eps, minpts, params=abx.Params(**kw)).cpu().numpy()
            tr = abx.profile_traversal()
        finally:
            abx.profile_enable(False)
        assert_same(lab, oracle.dbscan(p, eps, minpts), f"{kw} eps={eps}")
        if overflow:  # (at the small eps a minPts > 2 run has no core point, hence no query)
            assert tr["queries"] > 0 and tr["visits"] > 0, tr


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_many_uneven_segments(abx, seed):
    """Hundreds of segments of uneven size, each with its own eps and minPts
    (friends-of-friends and DBSCAN mixed in one call), must each equal the
    oracle on that segment alone."""
    rng = np.random.default_rng(100 + seed)
    sizes = np.concatenate([[0, 1, 2, 0], rng.integers(1, 3000, 300), rng.integers(3000, 40000, 8)])
    rng.shuffle(sizes)
    segs, eps, mp = [], [], []
    for k, n in enumerate(sizes):
        if n == 0:
            segs.append(np.zeros((0, 3), np.float32))
        else:
            p = _clumpy(rng, int(n), 4, 0.01)
            if k % 3 == 0:  # a segment far from the unit box, scaled
                p = (p * 50.0 - 20.0).astype(np.float32)
            segs.append(p)
        e = float(np.float32(rng.uniform(0.005, 0.03)))
        eps.append(e * (50.0 if k % 3 == 0 else 1.0))
        mp.append(int(rng.choice([1, 2, 3, 5, 10])))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    allp = torch.from_numpy(np.concatenate(segs).astype(np.float32)).cuda()
    lab = abx.dbscan_batch(allp, off, eps, mp)
    torch.cuda.synchronize()
    assert abx.device_status() == 0
    lab = lab.cpu().numpy()
    for k in range(len(sizes)):
        want = oracle.dbscan(segs[k], eps[k], mp[k])
        assert_same(lab[off[k]:off[k + 1]], want, f"segment {k} (n={sizes[k]}, minPts={mp[k]})")


def test_batch_of_stream_requests(abx):
    """A batch shaped like the served stream: halo-like requests of
    log-uniform size, minPts in {2, 5, 10}, eps from the linking length."""
    from workloads import request_stream
    reqs = [r for r in request_stream(60, n_hi=2e5)]
    segs = [r.points() for r in reqs]
    off = np.concatenate([[0], np.cumsum([len(p) for p in segs])]).astype(np.int64)
    allp = torch.from_numpy(np.concatenate(segs)).cuda()
    lab = abx.dbscan_batch(allp, off, [r.eps for r in reqs], [r.minpts for r in reqs]).cpu().numpy()
    assert abx.device_status() == 0
    for k, r in enumerate(reqs):
        assert_same(lab[off[k]:off[k + 1]], oracle.dbscan(segs[k], r.eps, r.minpts), f"request {k}")


def test_sampled_bounds_large_input_with_outliers(abx):
    """Inputs of 2^22 points and more place the grid from a sample of the
    points; outliers the sample misses are clamped into the grid, which never
    changes a label; a non-finite coordinate anywhere is still reported."""
    rng = np.random.default_rng(21)
    n = (1 << 22) + 5
    p = clumps(n, 4000, 21, a0=0.002)
    far = rng.integers(0, n, 7)
    p[far] = np.array([[5.0, -3.0, 9.0]], np.float32) + rng.random((7, 3)).astype(np.float32) * 1e-4
    eps = float(np.float32(0.168 * n ** (-1 / 3)))
    assert_same(gpu_labels(abx, p, eps, 2), oracle.dbscan(p, eps, 2), "outliers")
    q = p.copy()
    q[n - 3, 2] = np.inf
    abx.dbscan(torch.from_numpy(q).cuda(), eps, 2)
    assert abx.device_status() == abx.ABX_ENONFINITE


def test_autotune_choice_is_used_and_labels_unchanged(abx, tmp_path):
    from paper_2409_10743_gb300 import autotune
    p = clumps(400_000, 400, 61, a0=0.02)
    eps = 0.003
    want = oracle.dbscan(p, eps, 5)
    t = torch.from_numpy(p).cuda()
    best = abx.autotune(t, eps, 5)
    assert best["leaf_size"] in (2, 4, 8) and best["block"] in (0, 128, 256, 512)
    assert abx.tune_get(len(p), 5) == best
    assert_same(abx.dbscan(t, eps, 5).cpu().numpy(), want, "tuned")
    path = str(tmp_path / "tune.json")
    autotune.save(path)
    abx.tune_set(len(p), 5, {"leaf_size": 2, "block": 128, "dense_cells": -1, "sub_bits": 0, "dense_min": 0})
    assert_same(abx.dbscan(t, eps, 5).cpu().numpy(), want, "set")
    assert autotune.load(path) >= 1 and abx.tune_get(len(p), 5) == best
    with pytest.raises(abx.AbxError):
        abx.tune_set(len(p), 5, {"leaf_size": 99})


@pytest.mark.parametrize("minpts", [2, 5])
def test_cluster_stats_match_oracle(abx, minpts):
    p = clumps(300_000, 300, 71, a0=0.02)
    eps = 0.004
    t = torch.from_numpy(p).cuda()
    lab = abx.dbscan(t, eps, minpts)
    s = abx.cluster_stats(t, lab)
    want = oracle.cluster_stats(p, lab.cpu().numpy())
    assert np.array_equal(s["ids"].cpu().numpy(), want["ids"])
    assert np.array_equal(s["sizes"].cpu().numpy(), want["sizes"])
    # centres: double sums in another order, rounded to float: within 1 ulp
    np.testing.assert_allclose(s["centres"].cpu().numpy(), want["centres"], rtol=1.2e-7, atol=0)
    np.testing.assert_allclose(s["radii"].cpu().numpy(), want["radii"], rtol=2e-6, atol=1e-7)


def test_pair_histogram_matches_oracle(abx):
    p = clumps(200_000, 200, 81, a0=0.02)
    edges = np.array([0.0, 0.001, 0.002, 0.004, 0.006, 0.01], np.float32)
    h = abx.BVH(torch.from_numpy(p).cuda(), leaf_size=4)
    got = h.pair_histogram(edges).cpu().numpy()
    h.close()
    assert np.array_equal(got, oracle.pair_histogram(p, edges))


@pytest.mark.parametrize("kw", [dict(dense_cells=-1), dict(dense_cells=-1, leaf_size=8), dict()],
                         ids=["dense-off", "dense-off-leaf8", "default"])
@pytest.mark.parametrize("minpts", [2, 6])
def test_key_widths(abx, kw, minpts):
    """Inputs large enough for the 32-bit key path: with dense cells off the grid
    resolves the point density (32-bit keys); with a coarse eps-relative grid
    the keys fit 32 bits too; otherwise 64-bit keys.  Labels never change."""
    for n, eps in [(150_000, 0.004), (200_000, 0.02)]:
        p = clumps(n, 100, n + minpts, a0=0.02)
        t = torch.from_numpy(p).cuda()
        abx.profile_enable(True)
        try:
            lab = abx.dbscan(t, eps, minpts, params=abx.Params(**kw)).cpu().numpy()
            bits = abx.profile_counters()["key_bits"]
        finally:
            abx.profile_enable(False)
        assert bits in (32, 64)
        assert_same(lab, oracle.dbscan(p, eps, minpts), f"{kw} n={n} key bits {bits}")
