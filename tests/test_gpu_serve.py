"""The serving loop: requests of very different sizes, submitted in a burst
and paced like arrivals, each come back exactly as abx_dbscan labels them
alone (and as the oracle does); the HBM budget, the queue bound, bounded
waits, host-injected allocation failures and shutdown behave as declared.
Failures are injected on the host (ABX_SERVE_FAULT), never on the GPU."""
import os
import time

import numpy as np
import pytest

import oracle
from workloads import request_stream

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10743_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def requests():
    reqs = request_stream(48, n_hi=3e5)
    return [(r, r.points()) for r in reqs]


def _alone(abx, p, eps, minpts):
    return abx.dbscan(torch.from_numpy(p).cuda(), eps, minpts).cpu().numpy()


@pytest.mark.parametrize("staging", ["0", "1"], ids=["from-caller-memory", "pinned-staging"])
def test_results_equal_alone_and_oracle(abx, requests, staging, monkeypatch):
    """Host-resident requests, their points copied straight from the caller's
    memory or staged through pinned buffers (ABX_SERVE_STAGING=1)."""
    monkeypatch.setenv("ABX_SERVE_STAGING", staging)
    srv = abx.Server(max_slots=2, max_batch_requests=16)
    try:
        tickets = [srv.submit(p, r.eps, r.minpts) for r, p in requests[:24]]   # a burst
        for r, p in requests[24:]:                                             # paced arrivals
            tickets.append(srv.submit(p, r.eps, r.minpts))
            time.sleep(0.002)
        for t, (r, p) in zip(tickets, requests):
            st, lab = srv.wait(t, 60000)
            assert st == abx.ABX_OK, abx.status_str(st)
            assert np.array_equal(lab, _alone(abx, p, r.eps, r.minpts)), f"request {r.k} differs from alone"
            assert np.array_equal(lab, oracle.dbscan(p, r.eps, r.minpts)), f"request {r.k} differs from oracle"
        s = srv.stats()
        assert s["completed"] == len(requests) and s["failed"] == 0
        assert s["batches"] < len(requests)          # requests were batched together
        assert s["p99_ms"] >= s["p50_ms"] > 0
    finally:
        srv.close()


def test_device_resident_requests(abx, requests):
    """In-situ requests already in HBM: labels come back on the device, equal
    to the alone-run, while host requests share the same batches."""
    srv = abx.Server(max_slots=2)
    try:
        ts = []
        for k, (r, p) in enumerate(requests[:20]):
            src = torch.from_numpy(p).cuda() if k % 2 == 0 else p
            ts.append((srv.submit(src, r.eps, r.minpts), r, p, k % 2 == 0))
        for t, r, p, dev in ts:
            st, lab = srv.wait(t, 60000)
            assert st == abx.ABX_OK
            got = lab.cpu().numpy() if dev else lab
            assert (lab.is_cuda if dev else isinstance(lab, np.ndarray))
            assert np.array_equal(got, _alone(abx, p, r.eps, r.minpts)), f"request {r.k}"
    finally:
        srv.close()


def test_budget_limits_admission(abx, requests):
    budget = 96 << 20
    srv = abx.Server(hbm_budget_bytes=budget, max_slots=3)
    try:
        big = np.random.default_rng(0).random((2_000_000, 3), dtype=np.float32)
        with pytest.raises(abx.AbxError) as e:
            srv.submit(big, 0.001, 2)
        assert e.value.code == abx.ABX_ENOMEM_BUDGET
        small = [(r, p) for r, p in requests if len(p) < 100_000][:12]
        ts = [srv.submit(p, r.eps, r.minpts) for r, p in small]
        for t, (r, p) in zip(ts, small):
            st, lab = srv.wait(t, 60000)
            assert st == 0 and np.array_equal(lab, oracle.dbscan(p, r.eps, r.minpts))
        assert 0 < srv.stats()["peak_bytes"] <= budget
    finally:
        srv.close()


def test_bounded_wait_queue_bound_and_shutdown(abx, requests, monkeypatch):
    monkeypatch.setenv("ABX_SERVE_FAULT", "hold")  # admit nothing
    srv = abx.Server(max_queue=2)
    try:
        r, p = requests[0]
        t1 = srv.submit(p, r.eps, r.minpts)
        srv.submit(p, r.eps, r.minpts)
        with pytest.raises(abx.AbxError) as e:
            srv.submit(p, r.eps, r.minpts)
        assert e.value.code == abx.ABX_EBUSY
        t0 = time.time()
        st, lab = srv.wait(t1, 50)
        assert st == abx.ABX_ETIMEOUT and lab is None and time.time() - t0 < 5
        assert srv.stats()["queued"] == 2
    finally:
        t0 = time.time()
        srv.close()                                  # queued requests are cancelled, no hang
        assert time.time() - t0 < 10


def test_injected_allocation_failure(abx, requests, monkeypatch):
    monkeypatch.setenv("ABX_SERVE_FAULT", "alloc")
    srv = abx.Server()
    try:
        r, p = requests[1]
        st, lab = srv.wait(srv.submit(p, r.eps, r.minpts), 60000)
        assert st == abx.ABX_ENOMEM and lab is None
        assert srv.stats()["failed"] == 1
    finally:
        srv.close()
    monkeypatch.delenv("ABX_SERVE_FAULT")
    assert abx.device_status() == 0                 # the GPU never saw a fault


def test_invalid_tickets_and_arguments(abx):
    srv = abx.Server()
    try:
        assert srv.wait(123456, 0)[0] == abx.ABX_EINVAL
        with pytest.raises(abx.AbxError):
            srv.submit(np.zeros((4, 3), np.float32), -1.0, 2)
        t = srv.submit(np.zeros((0, 3), np.float32), 0.1, 2)
        assert srv.wait(t, 1000)[0] == abx.ABX_OK
    finally:
        srv.close()


def test_device_request_waits_for_its_producer_stream(abx):
    """Device points written by work still queued on another stream at submit
    time: the server must read them only after that work (the producer stream
    passed to submit), not whatever the buffer held before."""
    from workloads import clumps
    p = clumps(60_000, 40, 4711, a0=0.01)
    eps, minpts = 0.004, 3
    want = oracle.dbscan(p, eps, minpts)
    src = torch.from_numpy(p).cuda()
    dst = torch.zeros_like(src)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    srv = abx.Server(max_slots=2)
    try:
        with torch.cuda.stream(side):
            torch.cuda._sleep(100_000_000)  # a bounded spin (~50 ms) ahead of the copy
            dst.copy_(src)
        t = srv.submit(dst, eps, minpts, stream=side)
        st, lab = srv.wait(t, 60_000)
        assert st == 0, abx.status_str(st)
        assert np.array_equal(lab.cpu().numpy(), want)
    finally:
        srv.close()
        side.synchronize()
