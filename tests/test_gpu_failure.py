"""Failure detection on the device, without a GPU fault: a bounded device wait
that can never be satisfied gives up, records a timeout in the device status
word, and returns; the context stays usable and the next clustering call is
exact again."""
import numpy as np
import pytest

import oracle
from cases import _clumpy

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


@pytest.mark.parametrize("limit", [1, 100, 5000])
def test_lookback_wait_runs_out(abx, limit):
    s = abx._stream(None)
    rc = abx.lib().abx_selftest_wait_timeout(limit, s)
    assert rc == abx.ABX_OK, abx.status_str(rc)
    assert abx.device_status() == abx.ABX_ETIMEOUT
    assert abx.device_status() == abx.ABX_OK  # read once, then cleared
    # the context is intact: a clustering call right after is exact
    p = _clumpy(np.random.default_rng(limit), 20_000, 8, 0.01)
    lab = abx.dbscan(torch.from_numpy(p).cuda(), 0.01, 3)
    torch.cuda.synchronize()
    assert abx.device_status() == abx.ABX_OK
    assert np.array_equal(lab.cpu().numpy(), oracle.dbscan(p, 0.01, 3))


def test_selftest_arguments(abx):
    s = abx._stream(None)
    assert abx.lib().abx_selftest_wait_timeout(0, s) == abx.ABX_EINVAL
    assert abx.lib().abx_selftest_wait_timeout(1 << 25, s) == abx.ABX_EINVAL
