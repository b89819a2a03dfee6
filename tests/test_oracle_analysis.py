"""Pins for the oracle's consumers of a clustering: per-cluster statistics
(sizes, centres, farthest-member radii -- the galaxy circles of the paper's
HACC section) and the pair-distance histogram (the "find all pairs within a
radius, apply F" form of subsection "Pair traversal")."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import brute
import oracle
from cases import _clumpy


def test_cluster_stats_closed_form():
    # the 8 corners of a cube of half-side 0.25 around (1, 2, 3): centre exact,
    # radius = sqrt(3) * 0.25; plus a pair on the x axis and two noise points
    c = np.array([1.0, 2.0, 3.0])
    corners = np.array([[dx, dy, dz] for dx in (-0.25, 0.25) for dy in (-0.25, 0.25) for dz in (-0.25, 0.25)])
    pts = np.concatenate([[[9.0, 9.0, 9.0]], c + corners, [[5.0, 0.0, 0.0], [5.5, 0.0, 0.0]], [[-9.0, 0, 0]]])
    pts = pts.astype(np.float32)
    lab = np.array([-1] + [1] * 8 + [9, 9] + [-1], np.int32)
    s = oracle.cluster_stats(pts, lab)
    assert s["ids"].tolist() == [1, 9] and s["sizes"].tolist() == [8, 2]
    assert np.array_equal(s["centres"][0], np.float32(c)) and np.array_equal(s["centres"][1], [5.25, 0, 0])
    assert s["radii"][0] == np.float32(np.sqrt(np.float32(3 * 0.0625))) and s["radii"][1] == 0.25


def test_cluster_stats_against_numpy():
    p = _clumpy(np.random.default_rng(3), 4000, 10, 0.01)
    lab = oracle.dbscan(p, 0.02, 4)
    s = oracle.cluster_stats(p, lab)
    ids = np.unique(lab[lab >= 0])
    assert np.array_equal(s["ids"], ids)
    assert np.array_equal(s["sizes"], [(lab == i).sum() for i in ids])
    cen = np.array([p[lab == i].astype(np.float64).mean(0) for i in ids], np.float32)
    np.testing.assert_allclose(s["centres"], cen, rtol=2e-7, atol=0)
    rad = np.array([np.sqrt(np.max(((p[lab == i] - cen[k]) ** 2).sum(1))) for k, i in enumerate(ids)])
    np.testing.assert_allclose(s["radii"], rad, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("seed", range(3))
def test_pair_histogram_against_brute(seed):
    rng = np.random.default_rng(seed)
    p = _clumpy(rng, 1500, 6, 0.02)
    edges = [0.0, 0.005, 0.01, 0.02, 0.04, 0.08]
    assert np.array_equal(oracle.pair_histogram(p, edges), brute.pair_histogram(p, edges))


def test_pair_histogram_exact_edges_and_total():
    # a lattice of spacing 0.125: distances exactly on the edges go to the lower bin
    lat = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    p = (lat * 0.125).astype(np.float32)
    h = oracle.pair_histogram(p, [0.0, 0.125, 0.125 * np.sqrt(2) + 1e-6, 0.2])
    assert h[0] == 3 * 4 * 4 * 3 // 1  # axis-neighbour pairs: 3 axes * 16 lines * 3 gaps
    assert np.array_equal(h, brute.pair_histogram(p, [0.0, 0.125, 0.125 * np.sqrt(2) + 1e-6, 0.2]))
    q = _clumpy(np.random.default_rng(8), 1200, 5, 0.02)
    assert oracle.pair_histogram(q, [0.0, 0.03]).sum() == oracle.pair_count(q, 0.03)


def test_planted_histogram_mistake_is_caught(tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dbscan_oracle.c")).read()
    old = "if (d2 > h->e2[b] && d2 <= h->e2[b + 1]) {"
    assert src.count(old) == 1
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, "if (d2 >= h->e2[b] && d2 < h->e2[b + 1]) {"))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lat = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    p = np.ascontiguousarray((lat * 0.125).astype(np.float32))
    e = np.array([0.0, 0.125, 0.2], np.float32)
    h = np.zeros(2, np.int64)
    lib.oracle_pair_histogram(ctypes.c_void_p(p.ctypes.data), ctypes.c_int64(len(p)), ctypes.c_void_p(e.ctypes.data),
                              ctypes.c_int32(2), ctypes.c_void_p(h.ctypes.data))
    assert not np.array_equal(h, brute.pair_histogram(p, e))
