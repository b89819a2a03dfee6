"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/abx.h declares, and rejects bad arguments on the host (no GPU needed:
argument checks run before any CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "abx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(abx_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_10743_gb300 import binding
    return binding.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["abx_dbscan", "abx_dbscan_batch", "abx_bvh_build", "abx_device_status"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    from paper_2409_10743_gb300 import build
    so = build.build()
    assert os.path.exists(so)
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_status_strings(lib):
    from paper_2409_10743_gb300 import binding
    assert binding.status_str(0) == "ok"
    assert "invalid" in binding.status_str(binding.ABX_EINVAL)
    assert "internal" in binding.status_str(binding.ABX_EINTERNAL)


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2409_10743_gb300.binding import ABX_EINVAL, ABX_OK, Params
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: checks come first
    assert lib.abx_dbscan(fake, -1, 0.1, 2, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(fake, 10, -0.1, 2, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(fake, 10, float("nan"), 2, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(fake, 10, float("inf"), 2, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(fake, 10, 0.1, 0, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(null, 10, 0.1, 2, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(fake, 10, 0.1, 2, null, null) == ABX_EINVAL
    assert lib.abx_dbscan(fake, 2 ** 31, 0.1, 2, fake, null) == ABX_EINVAL
    assert lib.abx_dbscan(null, 0, 0.1, 2, null, null) == ABX_OK  # empty input: no-op
    bad = Params(leaf_size=33)
    assert lib.abx_dbscan_ex(fake, 10, 0.1, 2, fake, ctypes.byref(bad), null) == ABX_EINVAL
    bad = Params(block=100)
    assert lib.abx_dbscan_ex(fake, 10, 0.1, 2, fake, ctypes.byref(bad), null) == ABX_EINVAL
    bad = Params(dense_cells=2)
    assert lib.abx_dbscan_ex(fake, 10, 0.1, 2, fake, ctypes.byref(bad), null) == ABX_EINVAL
    for bad in (Params(schedule=3), Params(schedule=-1), Params(sort_digit_bits=9), Params(sort_digit_bits=10),
                Params(sort_digit_bits=12)):
        assert lib.abx_dbscan_ex(fake, 10, 0.1, 2, fake, ctypes.byref(bad), null) == ABX_EINVAL


def test_graph_arguments_rejected_on_host(lib):
    from paper_2409_10743_gb300.binding import ABX_EINVAL
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)
    h = ctypes.c_void_p()
    assert lib.abx_graph_create(fake, 10, 0.1, 2, fake, null, null) == ABX_EINVAL   # no handle
    assert lib.abx_graph_create(fake, 0, 0.1, 2, fake, null, ctypes.byref(h)) == ABX_EINVAL  # n = 0
    assert lib.abx_graph_create(fake, 10, -1.0, 2, fake, null, ctypes.byref(h)) == ABX_EINVAL
    assert lib.abx_graph_create(null, 10, 0.1, 2, fake, null, ctypes.byref(h)) == ABX_EINVAL
    assert lib.abx_graph_launch(null, null) == ABX_EINVAL
    assert lib.abx_graph_destroy(null) == ABX_EINVAL


def test_batch_arguments_rejected_on_host(lib):
    from paper_2409_10743_gb300.binding import ABX_EINVAL, ABX_OK
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)
    off = np.array([0, 5, 3], np.int64)  # decreasing
    eps = np.array([0.1, 0.1], np.float32)
    mp = np.array([2, 2], np.int32)
    assert lib.abx_dbscan_batch(fake, off.ctypes.data, 2, eps.ctypes.data, mp.ctypes.data, fake, null) == ABX_EINVAL
    off = np.array([1, 5, 9], np.int64)  # must start at 0
    assert lib.abx_dbscan_batch(fake, off.ctypes.data, 2, eps.ctypes.data, mp.ctypes.data, fake, null) == ABX_EINVAL
    off = np.array([0, 5, 9], np.int64)
    bad_mp = np.array([2, 0], np.int32)
    assert lib.abx_dbscan_batch(fake, off.ctypes.data, 2, eps.ctypes.data, bad_mp.ctypes.data, fake,
                                null) == ABX_EINVAL
    assert lib.abx_dbscan_batch(fake, null, 0, null, null, fake, null) == ABX_OK
    assert lib.abx_dbscan_batch(fake, null, -1, null, null, fake, null) == ABX_EINVAL


def test_bvh_arguments_rejected_on_host(lib):
    from paper_2409_10743_gb300.binding import ABX_EINVAL
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)
    h = ctypes.c_void_p()
    from paper_2409_10743_gb300.binding import Params
    assert lib.abx_bvh_build(fake, 0, None, ctypes.byref(h), null) == ABX_EINVAL
    assert lib.abx_bvh_build(fake, 10, ctypes.byref(Params(leaf_size=64)), ctypes.byref(h), null) == ABX_EINVAL
    assert lib.abx_bvh_build(fake, 10, ctypes.byref(Params(schedule=3)), ctypes.byref(h), null) == ABX_EINVAL
    assert lib.abx_bvh_build(fake, 10, ctypes.byref(Params(sort_digit_bits=9)), ctypes.byref(h), null) == ABX_EINVAL
    assert lib.abx_bvh_build(null, 10, None, ctypes.byref(h), null) == ABX_EINVAL
    assert lib.abx_bvh_count(null, fake, 1, 0.1, 1, fake, null) == ABX_EINVAL
    assert lib.abx_bvh_first_hit(null, fake, 1, 0.1, fake, null) == ABX_EINVAL
    assert lib.abx_bvh_destroy(null) == ABX_EINVAL


def test_no_cpu_fallback_in_the_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2409_10743_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
