"""Pins the oracle's periodic Delaunay triangulation.

A Delaunay triangle's circumcircle contains no other cell (Sussman, arXiv
1702.02939, Sec. 2.C.3).  Pins: brute-force empty-circle check in exact Python
integers over every periodic image, the Euler characteristic of the torus
(exactly 2N triangles, mean coordination exactly 6), agreement with Qhull on
tiled points, ring symmetry, and exactly degenerate lattices.
"""
import numpy as np
import pytest

import oracle
import workloads


def snapped(n, seed):
    x, y, th, L = workloads.spv_uniform(n, seed)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    return x, y, Lx, Ly, q


def to_int(v, q):
    return [int(round(float(t) * 2.0 ** q)) for t in v]


def incircle_int(a, b, c, d):
    rows = []
    for p in (a, b, c):
        dx, dy = p[0] - d[0], p[1] - d[1]
        rows.append((dx, dy, dx * dx + dy * dy))
    (a0, a1, a2), (b0, b1, b2), (c0, c1, c2) = rows
    return a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0)


def check_empty_circles(x, y, Lx, Ly, q, topo, strict_ok=False):
    X, Y = to_int(x, q), to_int(y, q)
    LX, LY = int(round(Lx * 2.0 ** q)), int(round(Ly * 2.0 ** q))
    n = len(X)
    images = [(X[k] + ox * LX, Y[k] + oy * LY) for k in range(n) for ox in (-1, 0, 1) for oy in (-1, 0, 1)]
    for i in range(n):
        m = topo.cnt[i]
        for a in range(m):
            b = (a + 1) % m
            j, k = topo.nbr[i, a], topo.nbr[i, b]
            pi = (X[i], Y[i])
            pj = (X[j] + int(topo.off[i, a, 0]) * LX, Y[j] + int(topo.off[i, a, 1]) * LY)
            pk = (X[k] + int(topo.off[i, b, 0]) * LX, Y[k] + int(topo.off[i, b, 1]) * LY)
            orient = (pj[0] - pi[0]) * (pk[1] - pi[1]) - (pj[1] - pi[1]) * (pk[0] - pi[0])
            assert orient > 0
            for p in images:
                if p in (pi, pj, pk):
                    continue
                assert incircle_int(pi, pj, pk, p) <= 0, (i, a)


def check_symmetric(topo):
    n = len(topo.cnt)
    for i in range(n):
        for a in range(topo.cnt[i]):
            j = topo.nbr[i, a]
            o = tuple(topo.off[i, a])
            back = [(topo.nbr[j, b], tuple(topo.off[j, b])) for b in range(topo.cnt[j])]
            assert (i, (-o[0], -o[1])) in back


@pytest.mark.parametrize("n,seed", [(16, 1), (32, 2), (64, 3)])
def test_brute_force_empty_circumcircles(n, seed):
    x, y, Lx, Ly, q = snapped(n, seed)
    topo = oracle.triangulate(x, y, Lx, Ly)
    check_empty_circles(x, y, Lx, Ly, q, topo)
    check_symmetric(topo)


@pytest.mark.parametrize("n", [16, 100, 400, 4096])
def test_euler_characteristic(n):
    x, y, Lx, Ly, q = snapped(n, 11)
    topo = oracle.triangulate(x, y, Lx, Ly)
    # torus: V - E + F = 0 with 3F = 2E  =>  F = 2N, sum of ring sizes = 6N
    assert int(topo.cnt.sum()) == 6 * n
    assert topo.cnt.mean() == 6.0
    check_symmetric(topo)


def test_matches_qhull_on_tiled_points():
    spatial = pytest.importorskip("scipy.spatial")
    n = 300
    x, y, Lx, Ly, q = snapped(n, 5)
    topo = oracle.triangulate(x, y, Lx, Ly)
    pts, ids = [], []
    for oy in (-1, 0, 1):
        for ox in (-1, 0, 1):
            for i in range(n):
                pts.append((x[i] + ox * Lx, y[i] + oy * Ly))
                ids.append((i, ox, oy))
    tri = spatial.Delaunay(np.array(pts))
    ours = set()
    for i in range(n):
        m = topo.cnt[i]
        for a in range(m):
            b = (a + 1) % m
            t = [(i, 0, 0), (int(topo.nbr[i, a]), *map(int, topo.off[i, a])),
                 (int(topo.nbr[i, b]), *map(int, topo.off[i, b]))]
            ours.add(frozenset(t))
    theirs = set()
    for s in tri.simplices:
        verts = [ids[v] for v in s]
        for c in verts:
            if c[1] == 0 and c[2] == 0:
                theirs.add(frozenset((v[0], v[1] - c[1], v[2] - c[2]) for v in verts))
    # every oracle triangle (in each central vertex's frame) is a Qhull triangle
    # and vice versa
    theirs_c = {t for t in theirs}
    ours_c = set()
    for t in ours:
        ours_c.add(t)
    assert ours_c == theirs_c


def test_square_lattice_degenerate_is_valid():
    """Every 4 lattice neighbours are exactly cocircular: the symbolic
    perturbation must still give a valid Delaunay triangulation."""
    x, y, L = workloads.square_lattice(6)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    topo = oracle.triangulate(x, y, Lx, Ly)
    assert int(topo.cnt.sum()) == 6 * len(x)
    check_empty_circles(x, y, Lx, Ly, q, topo)
    check_symmetric(topo)


def test_triangular_lattice_has_six_neighbours():
    x, y, Lx, Ly = workloads.triangular_lattice(6, 6)
    Lx, Ly, q = oracle.box(Lx, Ly)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    topo = oracle.triangulate(x, y, Lx, Ly)
    assert set(topo.cnt.tolist()) == {6}
    check_empty_circles(x, y, Lx, Ly, q, topo)


def test_plain_delaunay_matches_qhull():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(4)
    X = rng.integers(0, 1 << 40, 200)
    Y = rng.integers(0, 1 << 40, 200)
    cnt, nbr = oracle.delaunay_plain(X, Y)
    tri = spatial.Delaunay(np.stack([X, Y], 1).astype(float))
    theirs = {frozenset(map(int, s)) for s in tri.simplices}
    interior = {i for i in range(len(X)) if cnt[i] > 0}
    assert len(interior) > 150
    ours = set()
    for i in interior:
        m = cnt[i]
        for a in range(m):
            j, k = int(nbr[i, a]), int(nbr[i, (a + 1) % m])
            ours.add(frozenset((i, j, k)))
    assert ours <= theirs
    assert {t for t in theirs if t & interior} == ours
