"""ctypes binding of libabx.so: same names as the C ABI, argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ABX_OK = 0
ABX_EINVAL = -1
ABX_ENOMEM = -2
ABX_ENOMEM_BUDGET = -3
ABX_ECUDA = -4
ABX_ETIMEOUT = -5
ABX_ECANCELLED = -6
ABX_EBUSY = -7
ABX_ENONFINITE = -8
ABX_EINTERNAL = -9


class AbxError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_str(code)} ({code})" if what else f"{status_str(code)} ({code})")


class Params(ctypes.Structure):
    """abx_params: 0 in any field = library default; no field changes the labels."""
    _fields_ = [("leaf_size", ctypes.c_int32), ("dense_cells", ctypes.c_int32),
                ("sub_bits", ctypes.c_int32), ("block", ctypes.c_int32), ("dense_min", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("sort_digit_bits", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


PARAM_KEYS = ("leaf_size", "dense_cells", "sub_bits", "block", "dense_min", "schedule", "sort_digit_bits")


class ServeConfig(ctypes.Structure):
    """abx_serve_config: 0 in any field = default (40 GiB, 2 slots, 512 requests,
    2^25 points per batch, 2^20 queued)."""
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("max_batch_requests", ctypes.c_int32), ("max_batch_points", ctypes.c_int64),
                ("max_queue", ctypes.c_int32), ("device", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class ServeReport(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "failed", "cancelled", "batches",
                                               "queued", "bytes_in_use", "peak_bytes")] + \
               [(k, ctypes.c_double) for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "requests_per_s",
                                               "mean_batch_requests")]


_lock = threading.Lock()
_lib = None
_vp, _i64, _i32, _f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float

_SIGS = {
    "abx_status_str": (ctypes.c_char_p, [_i32]),
    "abx_dbscan": (_i32, [_vp, _i64, _f32, _i32, _vp, _vp]),
    "abx_dbscan_ex": (_i32, [_vp, _i64, _f32, _i32, _vp, ctypes.POINTER(Params), _vp]),
    "abx_dbscan_host": (_i32, [_vp, _i64, _f32, _i32, _vp, _vp]),
    "abx_graph_create": (_i32, [_vp, _i64, _f32, _i32, _vp, _vp, _vp]),
    "abx_graph_launch": (_i32, [_vp, _vp]),
    "abx_graph_destroy": (_i32, [_vp]),
    "abx_device_status": (_i32, [_vp]),
    "abx_selftest_wait_timeout": (_i32, [_i32, _vp]),
    "abx_dbscan_batch": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "abx_dbscan_batch_ex": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, ctypes.POINTER(Params), _vp]),
    "abx_autotune_batch": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, ctypes.POINTER(Params), _vp]),
    "abx_bvh_build": (_i32, [_vp, _i64, ctypes.POINTER(Params), ctypes.POINTER(_vp), _vp]),
    "abx_bvh_count": (_i32, [_vp, _vp, _i64, _f32, _i32, _vp, _vp]),
    "abx_bvh_first_hit": (_i32, [_vp, _vp, _i64, _f32, _vp, _vp]),
    "abx_bvh_info": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i32), _vp]),
    "abx_bvh_destroy": (_i32, [_vp]),
    "abx_profile_enable": (_i32, [_i32]),
    "abx_profile_stage_count": (_i32, []),
    "abx_profile_stage_name": (ctypes.c_char_p, [_i32]),
    "abx_profile_read": (_i32, [_vp, _i32]),
    "abx_launch_count": (ctypes.c_uint64, []),
    "abx_profile_counters": (_i32, [_vp, _i32]),
    "abx_profile_traversal": (_i32, [_vp, _i32]),
    "abx_cluster_stats": (_i32, [_vp, _vp, _i64, ctypes.POINTER(_i32), _vp, _vp, _vp, _vp, _vp]),
    "abx_bvh_pair_histogram": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "abx_bvh_pairs": (_i32, [_vp, _f32, ctypes.POINTER(_i64), _vp, _i64, ctypes.POINTER(_i64), _vp]),
    "abx_autotune": (_i32, [_vp, _i64, _f32, _i32, _vp, ctypes.POINTER(Params), _vp]),
    "abx_tune_get": (_i32, [_i64, _i32, ctypes.POINTER(Params)]),
    "abx_tune_set": (_i32, [_i64, _i32, ctypes.POINTER(Params)]),
    "abx_serve_create": (_i32, [ctypes.POINTER(ServeConfig), ctypes.POINTER(_vp)]),
    "abx_serve_submit": (_i32, [_vp, _vp, _i64, _f32, _i32, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "abx_serve_wait": (_i32, [_vp, ctypes.c_uint64, _i32]),
    "abx_serve_stats": (_i32, [_vp, ctypes.POINTER(ServeReport)]),
    "abx_serve_destroy": (_i32, [_vp]),
}


def lib(path: str | None = None):
    """Load libabx.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or _build.build()
            if not os.path.exists(so):
                raise RuntimeError(f"abx CUDA library not found at {so}")
            L = ctypes.CDLL(so)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_str(code: int) -> str:
    return lib().abx_status_str(int(code)).decode()


def _check(rc: int, what: str):
    if rc != ABX_OK:
        raise AbxError(rc, what)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _points_dev(points):
    import torch
    if not isinstance(points, torch.Tensor) or not points.is_cuda:
        raise TypeError("points must be a CUDA torch tensor")
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
        raise TypeError("points must be float32 of shape (n, 3)")
    return points.contiguous()


def dbscan(points, eps: float, minpts: int, labels=None, params: Params | None = None, stream=None):
    """Cluster device points (torch float32 (n, 3) on CUDA) -> int32 labels on
    the same device (cluster id = smallest member index, noise = -1).
    Asynchronous on ``stream`` (default: torch's current stream)."""
    import torch
    p = _points_dev(points)
    n = p.shape[0]
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=p.device)
    s = _stream(stream)
    with torch.cuda.device(p.device):
        if params is None:
            rc = lib().abx_dbscan(p.data_ptr(), n, float(np.float32(eps)), int(minpts), labels.data_ptr(), s)
        else:
            rc = lib().abx_dbscan_ex(p.data_ptr(), n, float(np.float32(eps)), int(minpts), labels.data_ptr(),
                                     ctypes.byref(params), s)
    _check(rc, "abx_dbscan")
    return labels


class Graph:
    """abx_graph: the whole clustering of one fixed input (these device
    buffers, eps, minPts, parameters) captured as a CUDA graph; launch()
    replays it on the current contents of the points."""

    def __init__(self, points, eps: float, minpts: int, labels=None, params: Params | None = None):
        import torch
        self.points = _points_dev(points)
        n = self.points.shape[0]
        self.labels = labels if labels is not None else torch.empty(n, dtype=torch.int32, device=self.points.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.points.device):
            rc = lib().abx_graph_create(self.points.data_ptr(), n, float(np.float32(eps)), int(minpts),
                                        self.labels.data_ptr(), ctypes.byref(params) if params is not None else None,
                                        ctypes.byref(self._h))
        _check(rc, "abx_graph_create")

    def launch(self, stream=None):
        import torch
        with torch.cuda.device(self.points.device):
            _check(lib().abx_graph_launch(self._h, _stream(stream)), "abx_graph_launch")
        return self.labels

    def close(self):
        if self._h:
            _check(lib().abx_graph_destroy(self._h), "abx_graph_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dbscan_host(points: np.ndarray, eps: float, minpts: int, labels: np.ndarray | None = None, stream=None):
    """Host -> host clustering through abx_dbscan_host (copies inside, blocks)."""
    p = np.ascontiguousarray(points, dtype=np.float32)
    if p.ndim != 2 or p.shape[1] != 3:
        raise TypeError("points must be float32 of shape (n, 3)")
    if labels is None:
        labels = np.empty(p.shape[0], dtype=np.int32)
    rc = lib().abx_dbscan_host(p.ctypes.data, p.shape[0], float(np.float32(eps)), int(minpts),
                               labels.ctypes.data, _stream(stream))
    _check(rc, "abx_dbscan_host")
    return labels


def _segments(offsets, eps, minpts):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = off.size - 1
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, np.float32), (nseg,)), dtype=np.float32)
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(minpts, np.int32), (nseg,)), dtype=np.int32)
    return off, nseg, e, m


def dbscan_batch(points, offsets, eps, minpts, labels=None, params: Params | None = None, stream=None):
    """Cluster concatenated segments; labels are segment-local."""
    import torch
    p = _points_dev(points)
    off, nseg, e, m = _segments(offsets, eps, minpts)
    if labels is None:
        labels = torch.empty(p.shape[0], dtype=torch.int32, device=p.device)
    with torch.cuda.device(p.device):
        rc = lib().abx_dbscan_batch_ex(p.data_ptr(), off.ctypes.data, nseg, e.ctypes.data, m.ctypes.data,
                                       labels.data_ptr(), ctypes.byref(params) if params is not None else None,
                                       _stream(stream))
    _check(rc, "abx_dbscan_batch")
    return labels


def autotune_batch(points, offsets, eps, minpts, stream=None) -> dict:
    """Time candidate parameters on this batch; the winner is remembered for
    batches of its class (used by dbscan_batch and the server) and returned."""
    import torch
    p = _points_dev(points)
    off, nseg, e, m = _segments(offsets, eps, minpts)
    lab = torch.empty(p.shape[0], dtype=torch.int32, device=p.device)
    best = Params()
    rc = lib().abx_autotune_batch(p.data_ptr(), off.ctypes.data, nseg, e.ctypes.data, m.ctypes.data,
                                  lab.data_ptr(), ctypes.byref(best), _stream(stream))
    _check(rc, "abx_autotune_batch")
    return {k: getattr(best, k) for k in PARAM_KEYS}


def autotune(points, eps: float, minpts: int, stream=None) -> dict:
    """Time candidate parameters on this input; the winner is remembered for
    its size class and returned as a dict."""
    import torch
    p = _points_dev(points)
    lab = torch.empty(p.shape[0], dtype=torch.int32, device=p.device)
    best = Params()
    rc = lib().abx_autotune(p.data_ptr(), p.shape[0], float(np.float32(eps)), int(minpts), lab.data_ptr(),
                            ctypes.byref(best), _stream(stream))
    _check(rc, "abx_autotune")
    return {k: getattr(best, k) for k in PARAM_KEYS}


def tune_get(n: int, minpts: int):
    p = Params()
    return None if lib().abx_tune_get(int(n), int(minpts), ctypes.byref(p)) != ABX_OK else \
        {k: getattr(p, k) for k in PARAM_KEYS}


def tune_set(n: int, minpts: int, params: dict) -> None:
    _check(lib().abx_tune_set(int(n), int(minpts), ctypes.byref(Params(**params))), "abx_tune_set")


def cluster_stats(points, labels, stream=None) -> dict:
    """Per cluster (increasing id): ids, sizes, centres (k, 3), radii -- torch
    tensors on the points' device."""
    import torch
    p = _points_dev(points)
    lab = labels.contiguous()
    n = p.shape[0]
    dev = p.device
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    sizes = torch.empty(n, dtype=torch.int32, device=dev)
    cen = torch.empty((n, 3), dtype=torch.float32, device=dev)
    rad = torch.empty(n, dtype=torch.float32, device=dev)
    k = _i32()
    rc = lib().abx_cluster_stats(p.data_ptr(), lab.data_ptr(), n, ctypes.byref(k), ids.data_ptr(), sizes.data_ptr(),
                                 cen.data_ptr(), rad.data_ptr(), _stream(stream))
    _check(rc, "abx_cluster_stats")
    K = k.value
    return {"ids": ids[:K], "sizes": sizes[:K], "centres": cen[:K], "radii": rad[:K]}


def device_status(stream=None) -> int:
    """Wait for the stream; return and clear the device status word."""
    return int(lib().abx_device_status(_stream(stream)))


def profile_enable(on=True) -> None:
    """Record CUDA events at every stage boundary of each clustering call
    (on=2: also count the pair traversal's work, in a slower kernel)."""
    _check(lib().abx_profile_enable(int(on)), "abx_profile_enable")


def profile_traversal() -> dict:
    """Node visits, leaf visits, point tests, unions, queries of the pair
    traversal in the most recent profile-mode-2 call."""
    v = np.zeros(5, dtype=np.int64)
    _check(lib().abx_profile_traversal(v.ctypes.data, 5), "abx_profile_traversal")
    return dict(zip(["visits", "leaves", "tests", "unions", "queries"], map(int, v)))


def profile_read() -> dict:
    """Milliseconds per stage of the most recent profiled call."""
    L = lib()
    n = L.abx_profile_stage_count()
    ms = np.zeros(n, dtype=np.float32)
    _check(L.abx_profile_read(ms.ctypes.data, n), "abx_profile_read")
    return {L.abx_profile_stage_name(i).decode(): float(ms[i]) for i in range(n)}


def profile_counters() -> dict:
    """Radix passes, Morton bits per axis, dense on, cells, leaves, root of the
    most recent profiled call."""
    v = np.zeros(7, dtype=np.int64)
    _check(lib().abx_profile_counters(v.ctypes.data, 7), "abx_profile_counters")
    return dict(zip(["radix_passes", "morton_bits", "dense_on", "dense_cells", "leaves", "root", "key_bits"],
                    map(int, v)))


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().abx_launch_count())


class BVH:
    """abx_bvh handle: build over device points, early-terminated counts and
    first hits, pair-distance histograms."""

    def __init__(self, points, leaf_size: int = 0, stream=None, params: Params | None = None):
        p = _points_dev(points)
        self._h = ctypes.c_void_p()
        self._stream = _stream(stream)
        self._points = p  # the build reads the points asynchronously
        if params is None:
            params = Params(leaf_size=int(leaf_size))
        rc = lib().abx_bvh_build(p.data_ptr(), p.shape[0], ctypes.byref(params), ctypes.byref(self._h),
                                 self._stream)
        _check(rc, "abx_bvh_build")

    def count(self, queries, eps: float, cap: int, out=None):
        import torch
        q = _points_dev(queries)
        if out is None:
            out = torch.empty(q.shape[0], dtype=torch.int32, device=q.device)
        rc = lib().abx_bvh_count(self._h, q.data_ptr(), q.shape[0], float(np.float32(eps)), int(cap),
                                 out.data_ptr(), self._stream)
        _check(rc, "abx_bvh_count")
        return out

    def first_hit(self, queries, eps: float, out=None):
        """Original index of one tree point within eps of each query (the
        first the traversal meets), -1 where there is none."""
        import torch
        q = _points_dev(queries)
        if out is None:
            out = torch.empty(q.shape[0], dtype=torch.int32, device=q.device)
        rc = lib().abx_bvh_first_hit(self._h, q.data_ptr(), q.shape[0], float(np.float32(eps)), out.data_ptr(),
                                     self._stream)
        _check(rc, "abx_bvh_first_hit")
        return out

    def pair_histogram(self, r_edges):
        """hist[b] = unordered pairs with fl(r_b^2) < d2 <= fl(r_{b+1}^2)."""
        import torch
        e = np.ascontiguousarray(r_edges, dtype=np.float32)
        h = torch.empty(e.size - 1, dtype=torch.int64, device="cuda")
        rc = lib().abx_bvh_pair_histogram(self._h, e.ctypes.data, e.size - 1, h.data_ptr(), self._stream)
        _check(rc, "abx_bvh_pair_histogram")
        return h

    def pairs_chunk(self, eps: float, cursor: int, out):
        """One call of abx_bvh_pairs: (status, new cursor, pairs written) into
        out, a CUDA int32 tensor of shape (cap, 2)."""
        cur = ctypes.c_int64(int(cursor))
        wrote = ctypes.c_int64(0)
        rc = lib().abx_bvh_pairs(self._h, float(np.float32(eps)), ctypes.byref(cur),
                                 out.data_ptr() if out.numel() else None, out.shape[0], ctypes.byref(wrote),
                                 self._stream)
        return rc, int(cur.value), int(wrote.value)

    def pairs(self, eps: float, cap: int = 1 << 22):
        """Every unordered neighbour pair once, as an (m, 2) int32 CUDA tensor
        of original indices with i < j, in the library's fixed order."""
        import torch
        out = torch.empty((cap, 2), dtype=torch.int32, device=self._points.device)
        parts, cursor, n = [], 0, self._points.shape[0]
        while cursor < n:
            rc, cursor, wrote = self.pairs_chunk(eps, cursor, out)
            if rc == ABX_ENOMEM:  # one point has more pairs than the buffer holds
                out = torch.empty((2 * out.shape[0], 2), dtype=torch.int32, device=out.device)
                continue
            _check(rc, "abx_bvh_pairs")
            parts.append(out[:wrote].clone())
        return torch.cat(parts) if parts else out[:0].clone()

    def info(self):
        n, L, lev = _i64(), _i64(), _i32()
        _check(lib().abx_bvh_info(self._h, ctypes.byref(n), ctypes.byref(L), ctypes.byref(lev), self._stream),
               "abx_bvh_info")
        return {"n_points": n.value, "n_leaves": L.value, "levels": lev.value}

    def close(self):
        if self._h:
            _check(lib().abx_bvh_destroy(self._h), "abx_bvh_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """abx_server: submit host point sets, wait for their labels.  The points
    and label arrays of a request are kept alive here until it is waited for."""

    def __init__(self, **cfg):
        c = ServeConfig(**cfg)
        self._h = ctypes.c_void_p()
        _check(lib().abx_serve_create(ctypes.byref(c), ctypes.byref(self._h)), "abx_serve_create")
        self._keep = {}

    def submit(self, points, eps: float, minpts: int, stream=None) -> int:
        """points: a numpy (n, 3) float32 array (host request) or a CUDA torch
        tensor (device request); the labels come back on the same side.  For a
        device request the server reads the points after the work enqueued so
        far on `stream` (default: torch's current stream), which produced them."""
        producer = None
        if hasattr(points, "is_cuda") and points.is_cuda:
            import torch
            p = _points_dev(points)
            lab = torch.empty(p.shape[0], dtype=torch.int32, device=p.device)
            pp, lp = p.data_ptr(), lab.data_ptr()
            producer = _stream(stream)
        else:
            p = np.ascontiguousarray(points, dtype=np.float32)
            if p.ndim != 2 or p.shape[1] != 3:
                raise TypeError("points must be float32 of shape (n, 3)")
            lab = np.empty(p.shape[0], dtype=np.int32)
            pp, lp = p.ctypes.data, lab.ctypes.data
        t = ctypes.c_uint64()
        rc = lib().abx_serve_submit(self._h, pp, p.shape[0], float(np.float32(eps)), int(minpts), lp, producer,
                                    ctypes.byref(t))
        _check(rc, "abx_serve_submit")
        self._keep[t.value] = (p, lab)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(status, labels): status ABX_OK with the labels, ABX_ETIMEOUT (ticket
        still pending), or the request's error."""
        rc = lib().abx_serve_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms))
        if rc == ABX_ETIMEOUT:
            return rc, None
        _, lab = self._keep.pop(ticket, (None, None))
        return rc, (lab if rc == ABX_OK else None)

    def stats(self) -> dict:
        r = ServeReport()
        _check(lib().abx_serve_stats(self._h, ctypes.byref(r)), "abx_serve_stats")
        return {k: getattr(r, k) for k, _ in ServeReport._fields_}

    def close(self):
        if self._h:
            _check(lib().abx_serve_destroy(self._h), "abx_serve_destroy")
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
