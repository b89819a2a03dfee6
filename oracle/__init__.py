"""Oracle for density-based clustering: plain CPU DBSCAN in C.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
(``paper_2409_10743_gb300``) never imports it, and the two share no code.

``dbscan`` computes the plain definition of DBSCAN from the paper's
"DBSCAN algorithm" subsection (eps-neighbourhood with the point itself, core
iff ``|N_eps| >= minPts``, clusters = components of the core points, border
points attached to a neighbouring cluster, the rest noise) with the exactness
contract written at the top of ``dbscan_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dbscan_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

# -ffp-contract=off: every float operation of the predicate is rounded on its
# own (GCC contracts a*b+c into an FMA by default on aarch64).
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_dbscan.restype = ctypes.c_int
            lib.oracle_dbscan.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                          ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_core_flags.restype = ctypes.c_int
            lib.oracle_core_flags.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                              ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_pair_count.restype = ctypes.c_int64
            lib.oracle_pair_count.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float]
            lib.oracle_pair_list.restype = ctypes.c_int64
            lib.oracle_pair_list.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p,
                                             ctypes.c_int64]
            lib.oracle_cluster_stats.restype = ctypes.c_int64
            lib.oracle_cluster_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64] + \
                [ctypes.c_void_p] * 4
            lib.oracle_pair_histogram.restype = ctypes.c_int
            lib.oracle_pair_histogram.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                  ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_pred.restype = ctypes.c_int
            lib.oracle_pred.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


_ERRORS = {-1: "invalid argument", -2: "non-finite coordinate", -3: "out of memory"}


def _points(points) -> np.ndarray:
    p = np.ascontiguousarray(points, dtype=np.float32)
    if p.ndim != 2 or p.shape[1] != 3:
        raise ValueError("points must be an (n, 3) array")
    return p


def dbscan(points, eps: float, minpts: int) -> np.ndarray:
    """Labels (int32): smallest original index of the point's cluster, -1 for noise."""
    p = _points(points)
    n = p.shape[0]
    labels = np.empty(n, dtype=np.int32)
    rc = _load().oracle_dbscan(p.ctypes.data, n, float(np.float32(eps)), int(minpts),
                               labels.ctypes.data)
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, f"error {rc}"))
    return labels


def core_flags(points, eps: float, minpts: int) -> np.ndarray:
    """core[i] = |N_eps(i)| >= minPts (bool)."""
    p = _points(points)
    n = p.shape[0]
    core = np.zeros(n, dtype=np.uint8)
    rc = _load().oracle_core_flags(p.ctypes.data, n, float(np.float32(eps)), int(minpts),
                                   core.ctypes.data)
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, f"error {rc}"))
    return core.astype(bool)


def pair_count(points, eps: float) -> int:
    """Number of unordered neighbour pairs {i, j}, i != j."""
    p = _points(points)
    r = _load().oracle_pair_count(p.ctypes.data, p.shape[0], float(np.float32(eps)))
    if r < 0:
        raise OracleError(_ERRORS.get(int(r), f"error {r}"))
    return int(r)


def pairs(points, eps: float) -> np.ndarray:
    """Every unordered neighbour pair as rows (i, j), i < j, original indices,
    sorted (int64, shape (m, 2))."""
    p = _points(points)
    total = pair_count(p, eps)
    out = np.zeros((max(total, 1), 2), dtype=np.int64)
    r = _load().oracle_pair_list(p.ctypes.data, p.shape[0], float(np.float32(eps)), out.ctypes.data, total)
    if r < 0:
        raise OracleError(_ERRORS.get(int(r), f"error {r}"))
    out = out[:total]
    return out[np.lexsort((out[:, 1], out[:, 0]))]


def pred(p, q, eps: float) -> bool:
    """The exact FP32 neighbour predicate on two points."""
    a = np.ascontiguousarray(p, dtype=np.float32).reshape(3)
    b = np.ascontiguousarray(q, dtype=np.float32).reshape(3)
    return bool(_load().oracle_pred(a.ctypes.data, b.ctypes.data, float(np.float32(eps))))


def cluster_stats(points, labels) -> dict:
    """Per cluster (increasing id): ids, sizes, centres (k, 3), radii."""
    p = _points(points)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    n = p.shape[0]
    ids = np.empty(n, np.int32)
    sizes = np.empty(n, np.int32)
    cen = np.empty((n, 3), np.float32)
    rad = np.empty(n, np.float32)
    k = _load().oracle_cluster_stats(p.ctypes.data, lab.ctypes.data, n, ids.ctypes.data, sizes.ctypes.data,
                                     cen.ctypes.data, rad.ctypes.data)
    if k < 0:
        raise OracleError(_ERRORS.get(int(k), f"error {k}"))
    return {"ids": ids[:k], "sizes": sizes[:k], "centres": cen[:k], "radii": rad[:k]}


def pair_histogram(points, r_edges) -> np.ndarray:
    """hist[b] = unordered pairs with fl(r_b^2) < d2 <= fl(r_{b+1}^2)."""
    p = _points(points)
    e = np.ascontiguousarray(r_edges, dtype=np.float32)
    h = np.zeros(e.size - 1, np.int64)
    rc = _load().oracle_pair_histogram(p.ctypes.data, p.shape[0], e.ctypes.data, e.size - 1, h.ctypes.data)
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, f"error {rc}"))
    return h
