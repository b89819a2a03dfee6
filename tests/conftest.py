import glob
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

GOLDEN_DIR = os.path.join(HERE, "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def _num(tok: str) -> float:
    t = tok.strip()
    return float.fromhex(t) if "0x" in t.lower() else float(t)


def load_golden(path: str):
    """Parse a golden case: returns (name, points float32 (n,3), eps, minpts, labels)."""
    eps = minpts = None
    pts, labels = [], None
    mode = None
    with open(path) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s.startswith("eps "):
                eps = _num(s.split()[1])
            elif s.startswith("minpts "):
                minpts = int(s.split()[1])
            elif s == "points":
                mode = "p"
            elif s == "labels":
                mode = "l"
            elif mode == "p":
                pts.append([_num(t) for t in s.split()])
            elif mode == "l":
                labels = [int(t) for t in s.split()]
    p = np.array(pts, dtype=np.float64)
    p32 = p.astype(np.float32)
    assert np.array_equal(p32.astype(np.float64), p), f"{path}: coordinates not exact in FP32"
    assert float(np.float32(eps)) == eps, f"{path}: eps not exact in FP32"
    assert labels is not None and len(labels) == len(pts)
    return os.path.basename(path), p32, float(eps), int(minpts), np.array(labels, dtype=np.int32)


def golden_cases():
    return [load_golden(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]


def has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def golden():
    return golden_cases()
