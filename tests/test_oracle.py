"""Pins for the oracle (CPU only).

The oracle is checked against things other than itself: the hand cases under
tests/golden (labels derived by hand from the paper's definitions), an
independent O(n^2) brute force from the definitions (tests/brute.py), the
friends-of-friends = connected-components identity, exact-arithmetic checks of
the FP32 predicate, invariants, and planted mistakes that the pins must catch.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import brute
import oracle
from conftest import golden_cases
from cases import _clumpy, _cases
from workloads import CONFIGS, clumps, uniform

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---- hand cases -------------------------------------------------------------

@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_golden_oracle(case):
    name, p, eps, minpts, want = case
    got = oracle.dbscan(p, eps, minpts)
    assert np.array_equal(got, want), f"{name}: {got} != {want}"


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_golden_brute(case):
    """The brute force agrees with the hand-derived labels too."""
    name, p, eps, minpts, want = case
    assert np.array_equal(brute.dbscan(p, eps, minpts), want), name


# ---- the predicate, by exact arithmetic ----------------------------------------

def _rn32(x: Fraction) -> Fraction:
    """Round an exact rational to the nearest FP32 (ties to even); values here
    are far from the subnormal range and fit a float64 exactly before rounding."""
    d = float(x)
    assert Fraction(d) == x, "intermediate not exact in float64"
    return Fraction(float(np.float32(d)))


def _pred_exact(p, q, eps) -> bool:
    P = [Fraction(float(v)) for v in np.asarray(p, np.float32)]
    Q = [Fraction(float(v)) for v in np.asarray(q, np.float32)]
    e = Fraction(float(np.float32(eps)))
    d = [_rn32(a - b) for a, b in zip(P, Q)]
    sq = [_rn32(v * v) for v in d]
    d2 = _rn32(_rn32(sq[0] + sq[1]) + sq[2])
    return d2 <= _rn32(e * e)


def test_fma_case_by_exact_arithmetic():
    case = [c for c in golden_cases() if c[0] == "fma_contraction.txt"][0]
    _, p, eps, _, _ = case
    assert _pred_exact(p[0], p[1], eps) is True
    assert _pred_exact(p[0], p[2], eps) is False
    assert oracle.pred(p[0], p[1], eps) is True
    assert oracle.pred(p[0], p[2], eps) is False


def test_pred_random_exact():
    rng = np.random.default_rng(11)
    for _ in range(3000):
        p = rng.random(3).astype(np.float32)
        q = (p + rng.normal(0, 0.3, 3)).astype(np.float32)
        eps = np.float32(rng.uniform(0.2, 0.6))
        assert oracle.pred(p, q, eps) == _pred_exact(p, q, eps)


# ---- brute force on small random inputs ---------------------------------------

@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_oracle_matches_brute(case):
    name, p, eps, minpts = case
    want = brute.dbscan(p, eps, minpts)
    got = oracle.dbscan(p, eps, minpts)
    assert np.array_equal(got, want), name
    assert np.array_equal(oracle.core_flags(p, eps, minpts), brute.core_flags(p, eps, minpts))
    assert oracle.pair_count(p, eps) == brute.pair_count(p, eps)


@pytest.mark.parametrize("seed", range(4))
def test_fof_equals_components(seed):
    """minPts = 2: labels are the connected components of the eps-graph, isolated
    points noise (subsection "Initial DBSCAN implementation")."""
    p = clumps(4000, 30, 900 + seed, a0=0.01)
    eps = 0.015
    assert np.array_equal(oracle.dbscan(p, eps, 2), brute.fof_components(p, eps))


@pytest.mark.slow
def test_c1_full_bruteforce():
    """The whole 32,768-point uniform FoF workload against the
    connected components of the brute-force eps-graph."""
    cfg = CONFIGS["fof-uniform-32K"]
    p = cfg.points()
    got = oracle.dbscan(p, cfg.eps, cfg.minpts)
    want = brute.fof_components(p, cfg.eps)
    assert np.array_equal(got, want)
    assert (got >= 0).sum() > 0


# ---- invariants ------------------------------------------------------------------

def _check_invariants(p, eps, minpts, lab):
    n = len(p)
    idx = np.arange(n)
    cl = lab >= 0
    assert np.all(lab[cl] <= idx[cl])                 # id = smallest member
    assert np.all(lab[lab[cl]] == lab[cl])            # the id point is in its cluster
    core = brute.core_flags(p, eps, minpts)
    assert np.all(cl[core])                           # every core point is clustered
    nb = brute.neighbour_lists(p, eps)
    for i in np.nonzero(~cl)[0]:                      # noise touches no core point
        assert not core[nb[i]].any()
    for i in np.nonzero(core)[0]:                     # core neighbours share a cluster
        cn = nb[i][core[nb[i]]]
        assert np.all(lab[cn] == lab[i])


@pytest.mark.parametrize("minpts", [2, 4, 8])
def test_invariants(minpts):
    p = _clumpy(np.random.default_rng(minpts), 1500, 10, 0.02)
    eps = 0.03
    _check_invariants(p, eps, minpts, oracle.dbscan(p, eps, minpts))


def _canonical(lab):
    """Partition as a set of frozensets (noise kept apart)."""
    groups = {}
    for i, l in enumerate(lab):
        groups.setdefault(int(l), set()).add(i)
    noise = frozenset(groups.pop(-1, set()))
    return noise, frozenset(frozenset(g) for g in groups.values())


@pytest.mark.parametrize("minpts", [2, 5])
def test_permutation_invariance(minpts):
    """FoF/core classification does not depend on input order; for minPts = 2
    the whole partition does not (for minPts > 2 a border point's choice can
    legitimately follow the indices, so only cores are compared there)."""
    rng = np.random.default_rng(5)
    p = _clumpy(rng, 1200, 8, 0.02)
    eps = 0.03
    perm = rng.permutation(len(p))
    a = oracle.dbscan(p, eps, minpts)
    b = oracle.dbscan(p[perm], eps, minpts)
    back = np.empty_like(b)
    back[perm] = b
    # map labels of the permuted run back to original indices of the id point
    relab = np.where(back >= 0, perm[np.clip(back, 0, None)], -1)
    if minpts == 2:
        assert _canonical(a) == _canonical(relab)
    else:
        core = oracle.core_flags(p, eps, minpts)
        assert _canonical(np.where(core, a, -1)) == _canonical(np.where(core, relab, -1))


@pytest.mark.parametrize("k", [-3, 2, 5])
def test_power_of_two_scaling(k):
    """Scaling coordinates and eps by 2^k is exact in FP32 (no overflow or
    underflow here), so the labels are identical."""
    p = _clumpy(np.random.default_rng(9), 1000, 6, 0.02)
    eps = 0.03
    s = np.float32(2.0 ** k)
    assert np.array_equal(oracle.dbscan(p, eps, 3), oracle.dbscan(p * s, eps * float(s), 3))


def test_exact_translation():
    """Translating points on a 2^-10 lattice by a multiple of 2^-10 keeps every
    difference exact, hence identical labels."""
    rng = np.random.default_rng(4)
    p = (rng.integers(0, 1024, (1500, 3)) / 1024.0).astype(np.float32)
    q = (p + np.float32(37 / 1024.0)).astype(np.float32)
    assert np.array_equal(q - np.float32(37 / 1024.0), p)
    eps = 0.02
    assert np.array_equal(oracle.dbscan(p, eps, 3), oracle.dbscan(q, eps, 3))


# ---- a closed form: the unit cubic lattice at eps = 1 ----------------------------------

def _lattice_expected(n, minpts, order):
    """Labels of the n^3 unit lattice at eps = 1, derived by hand: a point's
    neighbours are itself and its axis neighbours inside the lattice (the
    diagonal ones are sqrt(2) away), so |N| = 7 - (faces of the cube the
    point lies on).  minPts 2: one cluster.  minPts 7: the interior points
    are core and linked along the axes; a point on exactly one face touches
    the interior point behind it (a border point); edge and corner points
    touch only non-core points (noise).  Ids are the smallest member index
    in the given order."""
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    on_faces = ((g == 0) | (g == n - 1)).sum(1)
    if minpts == 2:
        member = np.ones(len(g), bool)
    else:
        assert minpts == 7
        member = on_faces <= 1
    want = np.full(len(g), -1, np.int32)
    pos = np.empty(len(g), np.int64)
    pos[order] = np.arange(len(g))            # index of lattice point k in the shuffled input
    want[member] = pos[member].min()
    return g, want, pos


@pytest.mark.parametrize("n,minpts", [(2, 2), (5, 2), (5, 7), (9, 7), (3, 7)])
def test_unit_lattice_closed_form(n, minpts):
    rng = np.random.default_rng(n * 10 + minpts)
    order = rng.permutation(n ** 3)
    g, want, pos = _lattice_expected(n, minpts, order)
    p = g[order].astype(np.float32)
    got = oracle.dbscan(p, 1.0, minpts)
    assert np.array_equal(got[pos], want)
    # just below 1 nothing is a neighbour: every point alone, hence noise
    below = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    assert (oracle.dbscan(p, below, 2) == -1).all()


@pytest.mark.parametrize("n,minpts", [(1, 1), (1, 2), (40, 40), (40, 41), (500, 7)])
def test_eps_beyond_the_diagonal(n, minpts):
    """eps = 2 exceeds the unit cube's diagonal: every pair is a neighbour pair,
    |N| = n for every point, so all points form one cluster with id 0 when
    n >= minPts and are all noise otherwise."""
    p = np.random.default_rng(n + minpts).random((n, 3), dtype=np.float32)
    want = np.zeros(n, np.int32) if n >= minpts else np.full(n, -1, np.int32)
    assert np.array_equal(oracle.dbscan(p, 2.0, minpts), want)


# ---- argument checking ---------------------------------------------------------------

def test_errors():
    p = np.zeros((4, 3), np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.dbscan(p, -1.0, 2)
    with pytest.raises(oracle.OracleError):
        oracle.dbscan(p, float("nan"), 2)
    with pytest.raises(oracle.OracleError):
        oracle.dbscan(p, 0.1, 0)
    q = p.copy()
    q[2, 1] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.dbscan(q, 0.1, 2)
    assert oracle.dbscan(np.zeros((0, 3), np.float32), 0.1, 2).shape == (0,)


# ---- planted mistakes: the pins must catch each one -------------------------------

MUTATIONS = [
    ("open neighbourhood", "return d2 <= e2;", "return d2 < e2;"),
    ("dropped z term", "    d2 = d2 + dz * dz;\n    return d2 <= e2;", "    d2 = d2 + 0.0f * dz;\n    return d2 <= e2;"),
    ("wrong sign in dy", "float dy = p[1] - q[1];\n    float dz = p[2] - q[2];\n    float d2 = dx * dx + dy * dy;\n"
     "    d2 = d2 + dz * dz;\n    return d2 <= e2;", "float dy = p[1] + q[1];\n    float dz = p[2] - q[2];\n"
     "    float d2 = dx * dx + dy * dy;\n    d2 = d2 + dz * dz;\n    return d2 <= e2;"),
    ("row offset off by one", "int64_t y = cy + (r % 3) - 1;", "int64_t y = cy + (r % 3);"),
    ("cell too small", "H *= 1.0 + ldexp(1.0, -10);", "H *= 0.5;"),
    ("core strict", "st.core[i] = st.count[i] >= minpts;", "st.core[i] = st.count[i] > minpts;"),
    ("border takes the largest K", "if (st->border[i] < 0 || k < st->border[i])",
     "if (st->border[i] < 0 || k > st->border[i])"),
    ("root is the larger index", "    if (a < b)\n        parent[b] = a;",
     "    if (a > b)\n        parent[b] = a;"),
    ("union of core with non-core", "if (j > i && st->core[j])", "if (j > i)"),
    ("border id ignored", "if (!st.core[i] && st.border[i] >= 0 && (int32_t)i < id[st.border[i]])",
     "if (0)"),
]


def _pins_pass(lib_dbscan) -> bool:
    for name, p, eps, minpts, want in golden_cases():
        if not np.array_equal(lib_dbscan(p, eps, minpts), want):
            return False
    for name, p, eps, minpts in _cases()[:12]:
        if not np.array_equal(lib_dbscan(p, eps, minpts), brute.dbscan(p, eps, minpts)):
            return False
    return True


def _mutated(mut, tmp_path):
    """The oracle with one planted mistake, as a labels(p, eps, minpts) call."""
    import ctypes
    name, old, new = mut
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dbscan_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor not found: {name}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_dbscan.restype = ctypes.c_int
    lib.oracle_dbscan.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_int32,
                                  ctypes.c_void_p]

    def run(p, eps, minpts):
        p = np.ascontiguousarray(p, np.float32)
        lab = np.empty(len(p), np.int32)
        rc = lib.oracle_dbscan(p.ctypes.data, len(p), float(np.float32(eps)), minpts, lab.ctypes.data)
        return lab if rc == 0 else None

    return run


@pytest.mark.parametrize("mut", MUTATIONS, ids=lambda m: m[0])
def test_planted_mistake_is_caught(mut, tmp_path):
    assert not _pins_pass(_mutated(mut, tmp_path)), f"planted mistake not caught: {mut[0]}"


# mistakes the lattice's closed form catches on its own (the other three do
# not change its labels: one cluster, and no core point next to a noise point)
LATTICE_CATCHES = ["open neighbourhood", "dropped z term", "wrong sign in dy", "row offset off by one",
                   "cell too small", "core strict", "border id ignored"]


@pytest.mark.parametrize("mut", [m for m in MUTATIONS if m[0] in LATTICE_CATCHES], ids=lambda m: m[0])
def test_lattice_closed_form_alone_catches(mut, tmp_path):
    run = _mutated(mut, tmp_path)
    for n, minpts in [(2, 2), (5, 2), (5, 7), (9, 7), (3, 7)]:
        order = np.random.default_rng(n * 10 + minpts).permutation(n ** 3)
        g, want, pos = _lattice_expected(n, minpts, order)
        got = run(g[order].astype(np.float32), 1.0, minpts)
        if got is None or not np.array_equal(got[pos], want):
            return
    raise AssertionError(f"the lattice's closed form missed: {mut[0]}")
