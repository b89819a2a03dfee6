"""GPU parity where the early exit of the rope walks is at its limit.

Every rope walk (the per-leaf candidate walk, the per-point counting and
border walks) stops at the first subtree it leaves whose Morton region holds
every grid cell a neighbour can fall in; the bound on how many cells two
neighbours can be apart comes from the neighbour test's rounding and the
quantisation's.  These inputs put neighbour pairs exactly at distance eps, on
cell boundaries, at several grid resolutions (the number of points sets the
Morton bits), offsets and scales, so that a bound one cell too small would
drop links and change labels.  Labels are compared with the oracle exactly.
"""
import numpy as np
import pytest

import oracle
from workloads import uniform

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


def labels_of(abx, p, eps, minpts, params=None):
    t = torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
    lab = abx.dbscan(t, eps, minpts, params=params)
    torch.cuda.synchronize()
    assert abx.device_status() == 0
    return lab.cpu().numpy()


def check(abx, p, eps, minpts, params=None, what=""):
    got = labels_of(abx, p, eps, minpts, params)
    want = oracle.dbscan(p, eps, minpts)
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{what}: {bad.size} labels differ, first {bad[:6]}")


def lattice(side, spacing, keep, seed, origin=(0.0, 0.0, 0.0)):
    """Lattice points k * spacing + origin (exact in FP32 for the values used),
    a random fraction `keep` of them, shuffled."""
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    p = g * spacing + np.asarray(origin)
    p = p[rng.random(len(p)) < keep]
    p32 = p.astype(np.float32)
    assert np.array_equal(p32.astype(np.float64), p)
    return p32[rng.permutation(len(p32))]


PARAMS = [None, dict(dense_cells=-1), dict(leaf_size=1, dense_cells=-1), dict(leaf_size=8, dense_cells=-1),
          dict(sub_bits=2), dict(schedule=2), dict(schedule=2, dense_cells=-1, leaf_size=2)]


@pytest.mark.parametrize("kw", PARAMS, ids=lambda k: "default" if k is None else
                         ",".join(f"{a}={b}" for a, b in k.items()))
@pytest.mark.parametrize("side,keep,minpts", [(40, 0.55, 2), (48, 0.8, 7), (24, 0.6, 3)])
def test_lattice_links_exactly_eps(abx, kw, side, keep, minpts):
    eps = 2.0 ** -6
    p = lattice(side, eps, keep, 100 + side + minpts)
    params = abx.Params(**kw) if kw else None
    check(abx, p, eps, minpts, params, f"side={side}")


@pytest.mark.parametrize("origin", [(0.5, 0.25, 0.125), (-3.0, 17.0, 1024.0), (1.0e4, -2.0e4, 3.0e4)])
def test_lattice_offsets(abx, origin):
    eps = 2.0 ** -4
    p = lattice(36, eps, 0.6, 7, origin)
    for minpts in (2, 5):
        for kw in (None, dict(dense_cells=-1, leaf_size=2)):
            check(abx, p, eps, minpts, abx.Params(**kw) if kw else None, f"origin={origin}")


@pytest.mark.parametrize("n,cells_per_eps", [(20_000, 0.3), (50_000, 1.0), (120_000, 2.5), (300_000, 0.15)])
def test_uniform_near_eps(abx, n, cells_per_eps):
    """Uniform points with eps a given number of grid cells (the dense-off grid
    has about 8 cells per point), so neighbours straddle cell boundaries at
    every offset."""
    p = uniform(n, 900 + n)
    b = 1
    while b < 21 and (1 << (3 * b)) < 8 * n:
        b += 1
    eps = float(np.float32(cells_per_eps / ((1 << b) - 1)))
    for minpts in (2, 4):
        check(abx, p, eps, minpts, abx.Params(dense_cells=-1), f"n={n} c={cells_per_eps}")
        check(abx, p, eps, minpts, None, f"n={n} c={cells_per_eps} dense")


def test_outliers_outside_sampled_bounds(abx):
    """Above 2^22 points the grid is placed from a 1/32 sample; points outside
    it are clamped into the edge cells.  Pairs among far outliers and across
    the clamp still have to be found."""
    n = (1 << 22) + 4096
    p = uniform(n, 4242)
    rng = np.random.default_rng(5)
    idx = rng.choice(n, 64, replace=False)
    eps = float(np.float32(0.168 / n ** (1 / 3)))
    # chains of outliers beyond the unit box, links exactly representable
    base = np.array([1.5, -0.75, 2.0], np.float32)
    step = np.float32(2.0 ** -12)
    for k, i in enumerate(idx):
        p[i] = base + np.float32(k) * np.array([step, 0, 0], np.float32)
    check(abx, p, float(np.float32(2.0 ** -12)), 2, abx.Params(dense_cells=-1), "outliers")
    check(abx, p, eps, 2, None, "outliers dense")


def test_batch_schedules_and_batch_tuner(abx):
    """Uneven segments, FoF and DBSCAN mixed: both traversal schedules, and
    the batch autotuner's pick (remembered for the class and used when no
    parameters are given), give every segment the oracle's labels."""
    from workloads import clumps
    rng = np.random.default_rng(31)
    sizes = [int(x) for x in np.exp(rng.uniform(np.log(200), np.log(60_000), 40))]
    segs = [clumps(n, max(1, n // 800), 700 + k, a0=0.01) for k, n in enumerate(sizes)]
    eps = [float(np.float32(0.168 / n ** (1 / 3))) for n in sizes]
    mp = [int(x) for x in rng.choice([2, 5, 10], len(sizes))]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    t = torch.from_numpy(np.concatenate(segs)).cuda()
    want = np.concatenate([oracle.dbscan(p, e, m) for p, e, m in zip(segs, eps, mp)])
    for kw in (dict(schedule=1), dict(schedule=2), dict(schedule=2, leaf_size=8, dense_cells=-1)):
        got = abx.dbscan_batch(t, off, eps, mp, params=abx.Params(**kw))
        torch.cuda.synchronize()
        assert abx.device_status() == 0
        assert np.array_equal(got.cpu().numpy(), want), kw
    best = abx.autotune_batch(t, off, eps, mp)
    assert best["schedule"] in (1, 2)
    got = abx.dbscan_batch(t, off, eps, mp)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("kw", [dict(leaf_size=1, dense_cells=-1), dict(leaf_size=2, dense_cells=-1), dict(leaf_size=4)],
                         ids=["leaf1", "leaf2", "dense-leaf4"])
@pytest.mark.parametrize("minpts", [3, 12, 40])
def test_dbscan_count_from_lists_and_list_overflow(abx, kw, minpts):
    """The core count first counts the own leaf and the listed candidate
    leaves and walks from the root only when they hold fewer than minPts
    neighbours; the union walks on where a list overflowed.  Over this range
    of eps (from a few clustered points to 90%) the lists run from empty to
    overflowing and the count from settled by the lists to needing the walk."""
    from workloads import clumps
    p = clumps(40_000, 30, 913 + minpts, a0=0.004)
    for eps in (0.002, 0.005, 0.012, 0.03):
        check(abx, p, eps, minpts, abx.Params(schedule=1, **kw), f"{kw} eps={eps}")
    abx.profile_enable(2)
    try:
        labels_of(abx, p, 0.03, minpts, abx.Params(schedule=1, **kw))
        tr = abx.profile_traversal()
    finally:
        abx.profile_enable(False)
    assert tr["queries"] > 0 and tr["visits"] > 0, tr  # some lists overflowed
