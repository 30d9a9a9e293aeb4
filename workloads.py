"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module only draws random numbers and lays out simple lattices; it holds
none of the method's arithmetic (no snapping, triangulation, forces or noise).
Both the CUDA path and the oracle receive the arrays produced here.

Workloads follow the runs described for the SPV model (Sussman, arXiv
1702.02939, Sec. 3): cells at unit density in a periodic square box of side
L = sqrt(N), uniform random positions and directors.
"""
import math

import numpy as np


def spv_uniform(n, seed, L=None):
    """Uniform random positions in [0, L)^2 (L = sqrt(n) by default) and
    directors uniform in [0, 2 pi)."""
    L = math.sqrt(n) if L is None else L
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, n)
    y = rng.uniform(0.0, L, n)
    theta = rng.uniform(0.0, 2.0 * math.pi, n)
    return x, y, theta, L


def spv_uniform_rect(n, seed, Lx, Ly):
    """Uniform random positions in [0, Lx) x [0, Ly) and directors uniform in
    [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, Lx, n)
    y = rng.uniform(0.0, Ly, n)
    theta = rng.uniform(0.0, 2.0 * math.pi, n)
    return x, y, theta


def triangular_lattice(m_cols, m_rows, a=1.0, jitter=0.0, seed=0):
    """Regular triangular lattice (hexagonal Voronoi cells) of spacing a in a
    periodic box Lx = m_cols a, Ly = m_rows a sqrt(3)/2 (m_rows even)."""
    assert m_rows % 2 == 0
    h = a * math.sqrt(3.0) / 2.0
    xs, ys = [], []
    for r in range(m_rows):
        for c in range(m_cols):
            xs.append((c + 0.5 * (r % 2) + 0.25) * a)
            ys.append((r + 0.5) * h)
    x, y = np.array(xs), np.array(ys)
    if jitter:
        rng = np.random.default_rng(seed)
        x = x + rng.uniform(-jitter, jitter, len(x))
        y = y + rng.uniform(-jitter, jitter, len(y))
    return x, y, m_cols * a, m_rows * h


def square_lattice(m, a=1.0):
    """Square lattice: every 4 neighbouring points are exactly cocircular."""
    g = (np.arange(m) + 0.5) * a
    X, Y = np.meshgrid(g, g, indexing="xy")
    return X.ravel().copy(), Y.ravel().copy(), m * a


def replica_sizes(R, seed, n_min=256, n_max=16384):
    """Replica sizes log-uniform on [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), R))).astype(np.int64)


def replica_params(R, seed, p0_range=(3.6, 4.0), v0_range=(0.01, 0.5)):
    rng = np.random.default_rng(seed + 1)
    p0 = rng.uniform(*p0_range, R)
    v0 = rng.uniform(*v0_range, R)
    return p0, v0
