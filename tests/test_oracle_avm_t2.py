"""Pins the oracle's T2 transitions (cell removal) and per-cell preferred
areas in the active vertex model.

Sussman, arXiv 1702.02939, Sec. 2.A names T2 transitions (cell removal) among
the AVM's topological changes; the paper's code performs only T1s.  Reading
used here: a triangular cell whose area is below a threshold is removed and
its three vertices merge into one at their centroid; a dying cell is driven
there by its own preferred area A0_c (Eq. 1 with per-cell A0_c and
P0_c = p0_c sqrt(A0_c)).  Pins: forces equal finite differences of E with
per-cell A0; a removal leaves a valid degree-3 network that still tiles the
box (sum of areas = Lx Ly, V = 2 N over the remaining cells, 3N edges); the
kept vertex is the smallest of the three at their centroid (computed here
independently) and each neighbour loses exactly one vertex; without a
threshold the cell stays a triangle.
"""
import numpy as np
import pytest

import oracle
import workloads


def network(n, seed):
    x, y, th, L = workloads.spv_uniform(n, seed)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    return oracle.avm_build(x, y, Lx, Ly), th


def mimg(d, L):
    if d > 0.5 * L:
        d -= L
    elif d < -0.5 * L:
        d += L
    return d


def wrap(v, L):
    r = np.fmod(v, L)
    if r < 0.0:
        r += L
    if r >= L:
        r -= L
    return r + 0.0


def check_alive_network(net, p0=3.8, a0=1.0):
    """A valid degree-3 network over the cells left (cc > 0) that tiles the box."""
    n, V, R = net.n, net.V, oracle.MAX_RING
    vc, vn = net.vc.reshape(V, 3), net.vn.reshape(V, 3)
    free = vc[:, 0] < 0
    assert np.all(vc[free] == -1) and np.all(vn[free] == -1)
    alive = net.cc > 0
    assert int((~free).sum()) == 2 * int(alive.sum())
    for v in np.nonzero(~free)[0]:
        for s in range(3):
            w = vn[v, s]
            assert w >= 0 and not free[w] and v in vn[w]
            assert alive[vc[v, s]]
            assert vc[v, s] in vc[w] and vc[v, (s + 1) % 3] in vc[w]
    deg = np.bincount(vn[~free].ravel(), minlength=V)
    assert set(deg[~free].tolist()) == {3}
    cv = net.cv.reshape(n, R)
    for c in range(n):
        m = net.cc[c]
        if m == 0:
            assert np.all(cv[c] == -1)
            continue
        assert m >= 3
        for a in range(m):
            v, w = cv[c, a], cv[c, (a + 1) % m]
            assert c in vc[v] and w in vn[v]
    assert int(net.cc.sum()) == 3 * int((~free).sum())
    A = oracle.avm_forces(net, p0, A0=a0)[2]
    assert np.all(A[alive] > 0) and np.all(A[~alive] == 0.0)
    assert abs(A.sum() - net.Lx * net.Ly) <= 1e-10 * net.Lx * net.Ly


def test_per_cell_a0_forces_match_finite_differences():
    net, _ = network(100, 7)
    rng = np.random.default_rng(3)
    a0 = rng.uniform(0.3, 1.6, net.n)
    p0 = rng.uniform(3.5, 4.1, net.n)
    Fx, Fy, A, P, E = oracle.avm_forces(net, p0, A0=a0)
    # E written out per cell from the areas and perimeters
    E_direct = float(np.sum((A - a0) ** 2 + (P - p0 * np.sqrt(a0)) ** 2))
    assert abs(E - E_direct) <= 1e-12 * abs(E_direct)
    scale = max(np.abs(Fx).max(), np.abs(Fy).max())
    h = 1e-6
    for v in range(0, net.V, 11):
        for arr, F in ((net.hx, Fx), (net.hy, Fy)):
            arr[v] += h
            Ep = oracle.avm_forces(net, p0, A0=a0)[4]
            arr[v] -= 2 * h
            Em = oracle.avm_forces(net, p0, A0=a0)[4]
            arr[v] += h
            assert abs(-(Ep - Em) / (2 * h) - F[v]) <= 1e-6 * scale


def run_until_t2(net, th, a0, t2_area, max_steps=3000, thr=0.04):
    """Steps until the first T2; returns (state before that step, after it,
    theta before, step index)."""
    for k in range(max_steps):
        new, th2, t1, t2 = oracle.avm_step(net, th, 3.8, 0.02, seed=5, step=k, A0=a0, thr=thr, t2_area=t2_area,
                                            counts=True)
        if t2:
            return net, new, th, k, t2
        net, th = new, th2
    return None


def test_dying_cell_is_removed_by_a_t2():
    net, th = network(64, 11)
    dying = 9
    a0 = np.ones(net.n)
    a0[dying] = 0.0
    res = run_until_t2(net, th, a0, t2_area=0.01)
    assert res is not None, "the dying cell never reached the T2 threshold"
    before, after, th_before, k, t2 = res
    assert t2 == 1
    assert after.cc[dying] == 0 and np.all(after.cc[np.arange(net.n) != dying] >= 3)
    check_alive_network(after, a0=a0)
    # the same step without T2s: the dying cell is the small triangle there
    plain, _, _ = oracle.avm_step(before, th_before, 3.8, 0.02, seed=5, step=k, A0=a0, thr=0.04, t2_area=0.0)
    assert plain.cc[dying] == 3
    R = oracle.MAX_RING
    tri = [int(v) for v in plain.cv[dying * R:dying * R + 3]]
    vk = min(tri)
    Lx, Ly = plain.Lx, plain.Ly
    x0, y0 = plain.hx[tri[0]], plain.hy[tri[0]]
    dx1, dy1 = mimg(plain.hx[tri[1]] - x0, Lx), mimg(plain.hy[tri[1]] - y0, Ly)
    dx2, dy2 = mimg(plain.hx[tri[2]] - x0, Lx), mimg(plain.hy[tri[2]] - y0, Ly)
    assert dx1 * dy2 - dx2 * dy1 < 2 * 0.01
    assert after.hx[vk] == wrap(x0 + (dx1 + dx2) / 3.0, Lx)
    assert after.hy[vk] == wrap(y0 + (dy1 + dy2) / 3.0, Ly)
    for v in tri:
        if v != vk:
            assert np.all(after.vc[3 * v:3 * v + 3] == -1)
    # each of the three neighbours lost exactly one vertex; nothing else changed count
    nbrs = {int(c) for v in tri for c in plain.vc[3 * v:3 * v + 3]} - {dying}
    assert len(nbrs) == 3
    for c in range(net.n):
        if c == dying:
            continue
        assert after.cc[c] == plain.cc[c] - (1 if c in nbrs else 0)
    # the kept vertex joins the three neighbours and the three outer vertices
    assert set(after.vc[3 * vk:3 * vk + 3].tolist()) == nbrs


def test_without_a_threshold_the_cell_stays_a_triangle():
    net, th = network(64, 11)
    a0 = np.ones(net.n)
    a0[9] = 0.0
    for k in range(600):
        net, th, _ = oracle.avm_step(net, th, 3.8, 0.02, seed=5, step=k, A0=a0, thr=0.04)
    assert net.cc[9] == 3
    check_alive_network(net, a0=a0)


@pytest.mark.parametrize("seed", [2, 3])
def test_several_deaths_keep_a_valid_network(seed):
    net, th = network(100, seed)
    rng = np.random.default_rng(seed)
    a0 = np.ones(net.n)
    dying = rng.choice(net.n, 6, replace=False)
    a0[dying] = 0.0
    total = 0
    for k in range(1500):
        net, th, _, t2 = oracle.avm_step(net, th, 3.8, 0.05, seed=seed, step=k, A0=a0, thr=0.04, t2_area=0.01,
                                         counts=True)
        total += t2
    assert total == len(dying) == int((net.cc == 0).sum())
    assert set(np.nonzero(net.cc == 0)[0].tolist()) == set(dying.tolist())
    check_alive_network(net, a0=a0)
