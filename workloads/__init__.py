"""Seeded synthetic particle sets shaped like the paper's cosmology workloads.

This module only draws random points; it holds none of the clustering
arithmetic, and both the GPU library's tests/benchmarks and the CPU oracle's
tests take their inputs from here.

The paper's own benchmark (section "ArborX improvements": one rank of a HACC
gas simulation, about 37M dark-matter particles, eps = 0.042 from the linking
length b = 0.168 of the mean inter-particle spacing) is not available, so these
stand in for it:

* ``uniform``: points uniform in the unit cube.
* ``clumps``: a halo-like mixture.  A fraction of the points sits in Plummer
  spheres whose masses follow dN/dM ~ M^-1.9 on [20, 2e5] (inverse-CDF draw),
  point counts by largest-remainder rounding of the mass fractions, scale
  radius a = a0 * count^(1/3); the rest is uniform.  Points falling outside the
  unit cube are redrawn (a periodic-free box).
* ``blobs``: anisotropic Gaussian blobs (Haar-random rotation, per-axis sigma
  log-uniform in [0.001, 0.01]) plus uniform noise.

Every generator is a pure function of its arguments and seed
(``numpy.random.Generator(PCG64(seed))``) and returns an ``(n, 3)`` float32
array in a shuffled order (no accidental locality in the input order).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LINKING_LENGTH = 0.168


def linking_eps(n: int, volume: float = 1.0) -> float:
    """eps = b * (V / n)^(1/3) with b = 0.168 (the paper's footnote on eps)."""
    return float(np.float32(LINKING_LENGTH * (volume / n) ** (1.0 / 3.0)))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return rng.random((n, 3), dtype=np.float32)


def _power_law_masses(rng, k: int, slope: float = -1.9, mmin: float = 20.0, mmax: float = 2.0e5):
    a = 1.0 + slope  # exponent of the cumulative mass function
    u = rng.random(k)
    lo, hi = mmin ** a, mmax ** a
    return (lo + u * (hi - lo)) ** (1.0 / a)


def _largest_remainder(total: int, w: np.ndarray) -> np.ndarray:
    quota = total * w / w.sum()
    base = np.floor(quota).astype(np.int64)
    rem = total - int(base.sum())
    if rem > 0:
        order = np.argsort(-(quota - base), kind="stable")
        base[order[:rem]] += 1
    return base


def _plummer_offsets(rng, a: np.ndarray) -> np.ndarray:
    """Offsets from the clump centre for scale radii ``a`` (one per point)."""
    m = a.shape[0]
    u = rng.random(m)
    u = np.clip(u, 1e-12, 1.0 - 1e-12)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    d = rng.standard_normal((m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * r[:, None]


def clumps(n: int, n_clumps: int, seed: int, clump_frac: float = 0.6, a0: float = 0.002,
           a_scale: float = 1.0, stats: dict | None = None) -> np.ndarray:
    """Plummer-clump + uniform mixture in the unit box (halo-like FoF input)."""
    rng = _rng(seed)
    n_in = int(round(clump_frac * n))
    w = _power_law_masses(rng, n_clumps)
    counts = _largest_remainder(n_in, w)
    centres = rng.random((n_clumps, 3))
    a = a0 * a_scale * np.cbrt(counts.astype(np.float64))
    owner = np.repeat(np.arange(n_clumps), counts)
    out = np.empty((n, 3), dtype=np.float32)
    # clump points, redrawn until inside [0, 1)^3
    todo = np.arange(n_in)
    chunk = 1 << 22
    while todo.size:
        bad = []
        for s in range(0, todo.size, chunk):
            idx = todo[s:s + chunk]
            o = owner[idx]
            p = centres[o] + _plummer_offsets(rng, a[o])
            pf = p.astype(np.float32)
            ok = np.all((pf >= 0.0) & (pf < 1.0), axis=1)
            out[idx[ok]] = pf[ok]
            bad.append(idx[~ok])
        todo = np.concatenate(bad) if bad else np.empty(0, np.int64)
    out[n_in:] = rng.random((n - n_in, 3), dtype=np.float32)
    perm = rng.permutation(n)
    if stats is not None:
        stats.update(n_clumps=n_clumps, clump_points=n_in, max_count=int(counts.max()),
                     counts_over_2e5=int((counts > 200000).sum()))
    return out[perm]


def blobs(n: int, n_blobs: int, seed: int, blob_frac: float = 0.8,
          sigma_lo: float = 0.001, sigma_hi: float = 0.01) -> np.ndarray:
    """Anisotropic Gaussian blobs plus uniform noise (general-DBSCAN input)."""
    rng = _rng(seed)
    n_in = int(round(blob_frac * n))
    centres = rng.random((n_blobs, 3))
    g = rng.standard_normal((n_blobs, 3, 3))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]  # Haar rotation
    sig = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), (n_blobs, 3)))
    owner = rng.integers(0, n_blobs, n_in)
    out = np.empty((n, 3), dtype=np.float32)
    chunk = 1 << 22
    for s in range(0, n_in, chunk):
        o = owner[s:s + chunk]
        z = rng.standard_normal((o.size, 3)) * sig[o]
        out[s:s + o.size] = (centres[o] + np.einsum("nij,nj->ni", q[o], z)).astype(np.float32)
    out[n_in:] = rng.random((n - n_in, 3), dtype=np.float32)
    return out[rng.permutation(n)]


@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    n: int
    eps: float
    minpts: int
    kind: str
    seed: int
    n_groups: int = 0
    a_scale: float = 1.0

    def points(self) -> np.ndarray:
        if self.kind == "uniform":
            return uniform(self.n, self.seed)
        if self.kind == "clumps":
            return clumps(self.n, self.n_groups, self.seed, a_scale=self.a_scale)
        if self.kind == "blobs":
            return blobs(self.n, self.n_groups, self.seed)
        raise ValueError(self.kind)

    def describe(self) -> str:
        return (f"{self.name}: {self.kind} N={self.n} eps={self.eps:.9g} minPts={self.minpts}"
                + (f" groups={self.n_groups}" if self.n_groups else "")
                + (f" a_scale={self.a_scale:g}" if self.a_scale != 1.0 else ""))


def _cfg(name, n, minpts, kind, seed, groups=0, eps=None, a_scale=1.0):
    return Config(name, n, linking_eps(n) if eps is None else float(np.float32(eps)), minpts,
                  kind, seed, groups, a_scale)


CONFIGS = {
    # FoF, uniform, 32768 points
    "fof-uniform-32K": _cfg("fof-uniform-32K", 32768, 2, "uniform", 1001),
    # halo-like FoF, 2^24 points, 20,000 clumps
    "fof-clumps-16M": _cfg("fof-clumps-16M", 1 << 24, 2, "clumps", 1002, 20000),
    # general DBSCAN, 10^7 points in 5,000 blobs + 20% noise, minPts 10, eps 0.004
    "dbscan-blobs-10M": _cfg("dbscan-blobs-10M", 10_000_000, 10, "blobs", 1003, 5000, eps=0.004),
    # per-rank-scale FoF, 2^27 points, 50,000 clumps
    "fof-clumps-134M": _cfg("fof-clumps-134M", 1 << 27, 2, "clumps", 1004, 50000),
}
# Stress variants with clumps ten times more concentrated, so that dense
# cells and large halos appear (the literal clump mixtures are nearly uniform
# at the linking length).  Reported beside, never instead of, the literal ones.
CONFIGS["fof-halos-16M"] = _cfg("fof-halos-16M", 1 << 24, 2, "clumps", 1102, 20000, a_scale=0.1)
CONFIGS["fof-halos-134M"] = _cfg("fof-halos-134M", 1 << 27, 2, "clumps", 1104, 50000, a_scale=0.1)


def scaled(cfg: Config, n: int, seed: int | None = None) -> Config:
    """The same mixture at another size (eps follows the linking-length rule
    for the FoF mixtures; fixed-eps configs keep their eps)."""
    groups = max(1, round(cfg.n_groups * n / cfg.n)) if cfg.n_groups else 0
    eps = linking_eps(n) if cfg.kind != "blobs" else cfg.eps
    return Config(f"{cfg.name}@{n}", n, eps, cfg.minpts, cfg.kind,
                  cfg.seed if seed is None else seed, groups, cfg.a_scale)


@dataclasses.dataclass(frozen=True)
class Request:
    k: int
    arrival_s: float
    n: int
    eps: float
    minpts: int

    def points(self) -> np.ndarray:
        groups = max(1, round(20000 * self.n / (1 << 24)))
        return clumps(self.n, groups, 5000 + self.k)


def request_stream(n_requests: int = 2000, rate_hz: float = 200.0, seed: int = 5000,
                   n_lo: float = 1e3, n_hi: float = 1e7) -> list[Request]:
    """The served stream: Poisson arrivals, log-uniform sizes, minPts in {2, 5, 10}."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    ns = np.floor(10.0 ** rng.uniform(math.log10(n_lo), math.log10(n_hi), n_requests)).astype(int)
    mp = rng.choice(np.array([2, 5, 10]), n_requests)
    return [Request(k, float(t[k]), int(ns[k]), linking_eps(int(ns[k])), int(mp[k]))
            for k in range(n_requests)]
