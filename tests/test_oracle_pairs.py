"""Pins for the oracle's pair list (every unordered neighbour pair once, the
set the paper's pair traversal hands to its callback, subsection "Pair
traversal"): equal to the pairs of a brute-force O(n^2) adjacency in numpy
float32, on clumpy sets, exact lattices (distances exactly eps), duplicates
at eps = 0, and consistent with the pair count."""
import numpy as np
import pytest

import brute
import oracle
from cases import _clumpy


def brute_pairs(p, eps):
    out = []
    for i, nb in enumerate(brute.neighbour_lists(p, eps)):
        for j in nb:
            if j > i:
                out.append((i, int(j)))
    a = np.array(out, dtype=np.int64).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))] if len(a) else a


def lattice(side, spacing, keep, seed):
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    p = (g * spacing).astype(np.float32)
    return p[rng.random(len(p)) < keep]


CASES = [
    ("clumpy", lambda: _clumpy(np.random.default_rng(5), 2500, 8, 0.02), 0.03),
    ("uniform", lambda: np.random.default_rng(6).random((3000, 3)).astype(np.float32), 0.05),
    ("lattice-at-eps", lambda: lattice(9, 0.125, 0.8, 7), 0.125),
    ("lattice-diag", lambda: lattice(8, 0.125, 0.9, 8), float(np.float32(0.125 * np.sqrt(2)))),
    ("duplicates-eps0", lambda: np.repeat(np.random.default_rng(9).random((300, 3)).astype(np.float32), 3, 0),
     0.0),
]


@pytest.mark.parametrize("name,make,eps", CASES, ids=[c[0] for c in CASES])
def test_pair_list_equals_brute_force(name, make, eps):
    p = make()
    got = oracle.pairs(p, eps)
    want = brute_pairs(p, eps)
    assert got.shape == want.shape, name
    assert np.array_equal(got, want), name
    assert len(got) == oracle.pair_count(p, eps)
    if len(got):
        assert (got[:, 0] < got[:, 1]).all()


def test_pair_list_empty_and_isolated():
    assert oracle.pairs(np.zeros((0, 3), np.float32), 0.1).shape == (0, 2)
    far = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    assert oracle.pairs(far, 0.5).shape == (0, 2)
    assert oracle.pairs(far, 1.0).tolist() == [[0, 1], [0, 2]]
