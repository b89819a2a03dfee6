"""abx_dbscan_noalloc, the entry point for callers that cannot allocate device
memory (for example an analysis hook inside a simulation that keeps all of
the GPU's memory for itself): called through the C ABI twice in a row, its
labels must equal those of abx_dbscan on the same input (labels are integers:
exact equality).  This file is collected last so that a run stopping at the
first failure has already run everything else; it also passes on its own in
a fresh process."""
import ctypes

import numpy as np
import pytest

from cases import _clumpy

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10743_gb300 import binding
    L = binding.lib()
    f = L.abx_dbscan_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p]
    return L


def _noalloc(L, pts, eps, minpts):
    n = pts.shape[0]
    out = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.abx_dbscan_noalloc(pts.data_ptr(), n, float(np.float32(eps)), int(minpts), out.data_ptr(), s)
    assert rc == 0, rc
    return out


def _pooled(pts, eps, minpts):
    from paper_2409_10743_gb300 import binding
    return binding.dbscan(pts, eps, minpts)


def test_two_calls_match_the_pooled_entry_point(lib):
    rng = np.random.default_rng(2024)
    cases = [(_clumpy(rng, 65536, 20, 0.01), 0.01, 2),   # the largest accepted size, FoF
             (_clumpy(rng, 40000, 12, 0.01), 0.02, 5)]   # smaller, general minPts, after a larger call
    for p, eps, minpts in cases:
        t = torch.from_numpy(p).cuda()
        got = _noalloc(lib, t, eps, minpts)
        want = _pooled(t, eps, minpts)
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"n={len(p)} minPts={minpts}: labels differ"
        assert (got >= 0).any()


def test_rejects_inputs_above_capacity(lib):
    t = torch.zeros((65537, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(65537, dtype=torch.int32, device="cuda")
    rc = lib.abx_dbscan_noalloc(t.data_ptr(), 65537, 0.1, 2, out.data_ptr(), ctypes.c_void_p(0))
    assert rc == -1  # ABX_EINVAL, nothing enqueued
