"""Host-side pieces of bench.py (no GPU): the algorithmic-bytes table, the
kernel-source hash that decides whether a committed ncu traffic figure still
applies, and the oracle's served-stream baseline."""
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2409_10743_gb300 import build as pkg_build  # noqa: E402


def test_stage_bytes_table():
    n = 1 << 27
    c32 = {"radix_passes": 4, "leaves": 24183430, "key_bits": 32}
    c64 = dict(c32, key_bits=64)
    per_leaf = c32["leaves"] / n
    # sort: first pass key in, key + index out; then key + index both ways
    assert bench.stage_bytes("sort", c32, n) == pytest.approx(12 + 3 * 16)
    assert bench.stage_bytes("sort", c64, n) == pytest.approx(20 + 3 * 24)
    assert bench.stage_bytes("morton", c32, n) == 16 and bench.stage_bytes("morton", c64, n) == 20
    assert bench.stage_bytes("gather", c32, n) == 32  # perm 4 + point 12 + sorted float4 16
    assert bench.stage_bytes("union", c32, n) == pytest.approx(25 + 64 * per_leaf)
    assert bench.stage_bytes("candidates", c32, n) == pytest.approx(48 * per_leaf)
    assert bench.stage_bytes("no-such-stage", c32, n) == 0
    # bounds: every point below 2^22 points, every 32nd above
    assert bench.stage_bytes("bounds", c32, n) == pytest.approx(12 / 32)
    assert bench.stage_bytes("bounds", c32, 1 << 20) == 12
    # no dense-cell pass when dense cells are off
    assert bench.stage_bytes("cells", dict(c32, dense_on=0), n) == 0 and bench.stage_bytes("cells", c32, n) == 12
    names = ["bounds", "morton", "bucket", "sort", "gather", "cells", "leaves", "build", "candidates", "union",
             "finalize"]
    total = sum(bench.stage_bytes(k, c32, n) for k in names)
    assert 250 < total < 330  # the FoF step on the 2^27-point workload: about 275 B per point


def test_kernel_source_hash_follows_the_include_chain(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2409_10743_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(pkg_build, "CSRC", str(dst))
    h_sort = pkg_build.kernel_source_hash("k_sort.cu")
    h_cluster = pkg_build.kernel_source_hash("k_cluster.cu")
    assert h_sort == pkg_build.kernel_source_hash("k_sort.cu") and h_sort != h_cluster
    # a header the file does not include leaves its hash alone ...
    (dst / "scan.cuh").write_text((dst / "scan.cuh").read_text() + "\n// edit\n")
    assert pkg_build.kernel_source_hash("k_sort.cu") == h_sort
    # ... one it includes (through work.cuh) changes it, for every kernel file
    (dst / "abx_internal.cuh").write_text((dst / "abx_internal.cuh").read_text() + "\n// edit\n")
    assert pkg_build.kernel_source_hash("k_sort.cu") != h_sort
    assert pkg_build.kernel_source_hash("k_cluster.cu") != h_cluster


def test_traffic_figures_only_for_matching_sources(tmp_path, monkeypatch):
    import json
    prof = tmp_path / "profiles"
    prof.mkdir()
    good = pkg_build.kernel_source_hash("k_sort.cu")
    (prof / "ncu_traffic.json").write_text(json.dumps({"stages": {
        "gather": {"source": "k_sort.cu", "source_sha": good, "dram_bytes_per_point_launch": 100.0},
        "sort": {"source": "k_sort.cu", "source_sha": "0" * 16, "dram_bytes_per_point_launch": 50.0}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("gather") == 100.0
    assert bench.ncu_traffic("sort") is None      # taken on other sources
    assert bench.ncu_traffic("union") is None     # never captured


def test_served_cpu_baseline_counts_requests():
    from workloads import request_stream
    reqs = [r for r in request_stream(2000)[:60] if r.n < 20000][:6]
    assert reqs
    pts = [r.points() for r in reqs]
    out = bench.served_cpu_baseline(reqs, pts)
    assert out["kind"] == "oracle" and out["unit"] == "requests/s"
    assert out["value"] > 0 and out["cores"] == (os.cpu_count() or 1)
    assert f"{len(reqs)} requests" in out["sample"]
    assert np.isfinite(out["value"])
