"""abx_dbscan_noalloc, the entry point for callers that cannot allocate device
memory (for example an analysis hook inside a simulation that keeps all of
the GPU's memory for itself): called through the C ABI several times in a
row, its labels must equal the oracle's and those of abx_dbscan on the same
input (labels are integers: exact equality).  The sequence runs the largest
accepted size first and then smaller inputs, minPts = 1 (every point core)
and inputs of 1 and 33 points, so state left in the shared fixed workspace by
an earlier call would show.  Its device status word is reported by
abx_device_status.  This file is collected last so that a run stopping at the
first failure has already run everything else; it also passes on its own in
a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
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


def test_calls_in_a_row_match_the_oracle_and_the_pooled_entry_point(lib):
    from paper_2409_10743_gb300 import binding
    rng = np.random.default_rng(2024)
    cases = [(_clumpy(rng, 65536, 20, 0.01), 0.01, 2),   # the largest accepted size, FoF, 32-bit keys
             (_clumpy(rng, 40000, 12, 0.01), 0.02, 5),   # smaller, general minPts, 64-bit keys
             (_clumpy(rng, 5000, 6, 0.01), 0.01, 1),     # minPts = 1: every point core
             (_clumpy(rng, 1, 1, 0.01), 0.01, 1),        # a single point
             (_clumpy(rng, 33, 2, 0.001), 0.01, 2),      # a ragged few
             (_clumpy(rng, 65536, 30, 0.005), 0.008, 3)]  # the largest again, after the small ones
    for p, eps, minpts in cases:
        t = torch.from_numpy(p).cuda()
        got = _noalloc(lib, t, eps, minpts)
        want = _pooled(t, eps, minpts)
        torch.cuda.synchronize()
        assert binding.device_status() == 0
        g = got.cpu().numpy()
        assert np.array_equal(g, oracle.dbscan(p, eps, minpts)), f"n={len(p)} minPts={minpts}: oracle differs"
        assert np.array_equal(g, want.cpu().numpy()), f"n={len(p)} minPts={minpts}: pooled path differs"


def test_status_word_is_reported(lib):
    """A non-finite coordinate is a precondition violation: the call still
    returns, and abx_device_status reports (and clears) it."""
    from paper_2409_10743_gb300 import binding
    rng = np.random.default_rng(9)
    p = _clumpy(rng, 3000, 4, 0.01)
    p[17, 1] = np.nan
    _noalloc(lib, torch.from_numpy(p).cuda(), 0.01, 2)
    assert binding.device_status() == binding.ABX_ENONFINITE
    assert binding.device_status() == 0
    q = _clumpy(rng, 3000, 4, 0.01)
    got = _noalloc(lib, torch.from_numpy(q).cuda(), 0.01, 2)
    assert binding.device_status() == 0
    assert np.array_equal(got.cpu().numpy(), oracle.dbscan(q, 0.01, 2))


def test_rejects_inputs_above_capacity(lib):
    t = torch.zeros((65537, 3), dtype=torch.float32, device="cuda")
    out = torch.empty(65537, dtype=torch.int32, device="cuda")
    rc = lib.abx_dbscan_noalloc(t.data_ptr(), 65537, 0.1, 2, out.data_ptr(), ctypes.c_void_p(0))
    assert rc == -1  # ABX_EINVAL, nothing enqueued
