"""Persist the autotuner's per-device table (abx_autotune / abx_tune_get /
abx_tune_set) as JSON, keyed by GPU name, mode and size class."""
from __future__ import annotations

import json

from . import binding

MODES = {"fof": 2, "dbscan": 3}  # a minPts value of each mode


def table() -> dict:
    """Every remembered entry of the current device: {"fof:20": {...}, ...}."""
    out = {}
    for name, mp in MODES.items():
        for c in range(33):
            p = binding.tune_get(1 << c, mp)
            if p is not None:
                out[f"{name}:{c}"] = p
    return out


def save(path: str) -> None:
    import torch
    dev = torch.cuda.get_device_name()
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[dev] = table()
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def load(path: str) -> int:
    """Install the saved entries of the current GPU model; returns how many."""
    import torch
    with open(path) as f:
        data = json.load(f).get(torch.cuda.get_device_name(), {})
    for key, p in data.items():
        name, c = key.split(":")
        binding.tune_set(1 << int(c), MODES[name], p)
    return len(data)
