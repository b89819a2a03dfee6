"""Small seeded input cases shared by the oracle pins and the GPU parity tests:
uniform, clumpy, exact lattices (distances exactly eps), duplicates with
eps = 0, planar and collinear sets, a single point, offset coordinates, and
the halo-like mixture at small sizes."""
import numpy as np

from workloads import clumps


def _clumpy(rng, n, k, spread, noise_frac=0.3):
    c = rng.random((k, 3))
    own = rng.integers(0, k, n)
    p = c[own] + rng.normal(0, spread, (n, 3))
    m = int(noise_frac * n)
    p[:m] = rng.random((m, 3))
    return p.astype(np.float32)


def _cases():
    rng = np.random.default_rng(123)
    out = []
    for n, eps, minpts in [(500, 0.08, 2), (800, 0.06, 3), (1000, 0.05, 5), (700, 0.1, 10),
                           (300, 0.2, 1), (1500, 0.04, 4)]:
        out.append((f"uniform-{n}-{minpts}", rng.random((n, 3)).astype(np.float32), eps, minpts))
    for n, eps, minpts in [(1200, 0.02, 2), (1500, 0.03, 5), (2000, 0.025, 10), (900, 0.05, 3)]:
        out.append((f"clumpy-{n}-{minpts}", _clumpy(rng, n, 8, 0.02), eps, minpts))
    # duplicates and exact lattice spacings (distances exactly eps)
    lat = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    lat = (lat * 0.125).astype(np.float32)
    keep = rng.random(len(lat)) < 0.7
    out.append(("lattice-fof", lat[keep], 0.125, 2))
    out.append(("lattice-dbscan", lat[keep], 0.125, 5))
    out.append(("lattice-diag", lat[keep], float(np.float32(0.125 * np.sqrt(2))), 7))
    dup = rng.random((200, 3)).astype(np.float32)
    dup = np.concatenate([dup, dup[rng.integers(0, 200, 300)]])
    out.append(("duplicates-eps0", dup, 0.0, 2))
    out.append(("duplicates-eps0-m3", dup, 0.0, 3))
    out.append(("duplicates-small", dup, 0.03, 4))
    planar = rng.random((1000, 3)).astype(np.float32)
    planar[:, 2] = 0.5
    out.append(("planar", planar, 0.04, 3))
    line = np.zeros((400, 3), np.float32)
    line[:, 0] = np.sort(rng.random(400)).astype(np.float32)
    out.append(("line", line, 0.003, 2))
    one = np.array([[0.3, 0.2, 0.1]], np.float32)
    out.append(("single", one, 0.1, 1))
    out.append(("single-noise", one, 0.1, 2))
    # negative and large coordinates, off-centre box
    off = (rng.random((800, 3)) * 40 - 20).astype(np.float32)
    out.append(("offset", off, 1.6, 3))
    # the C-config mixtures at small sizes
    out.append(("clumps-mix", clumps(3000, 40, 77, a0=0.01), 0.02, 2))
    out.append(("clumps-mix-m5", clumps(3000, 40, 78, a0=0.01), 0.03, 5))
    return out
