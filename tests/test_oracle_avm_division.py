"""Pins the oracle's cell division in the active vertex model.

Sussman, arXiv 1702.02939, Sec. 2.A lists cell division among the features
vertex models add for living tissue; the paper's code has none.  Reading
used here: a cell divides along a line of a given direction through the mean
of its vertices; the two cut points become new vertices on the cut edges,
the cell keeps one side and a new cell (next free slot) takes the other.
Pins: the network stays a valid degree-3 tiling of the box (two vertices per
cell, sum of areas = Lx Ly); the two daughters' areas add up to the mother's
and their perimeters to the mother's plus twice the chord; the new vertices
lie on the mother's edges on opposite sides of the mean along the direction;
the neighbours across the cut edges keep their areas; dynamics (T1 and T2
passes) continue on the grown network.
"""
import numpy as np
import pytest

import oracle
import workloads
from test_oracle_avm_t2 import check_alive_network, mimg

R = oracle.MAX_RING


def grown(n, seed, cap):
    x, y, th, L = workloads.spv_uniform(n, seed)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    net = oracle.avm_build(x, y, Lx, Ly).with_capacity(cap)
    theta = np.concatenate([th, np.zeros(cap - n)])
    return net, theta, np.full(cap, 3.8), np.full(cap, 0.1), np.ones(cap)


def polygon(net, c):
    vs = [int(v) for v in net.cv[c * R:c * R + net.cc[c]]]
    x0, y0 = net.hx[vs[0]], net.hy[vs[0]]
    return vs, np.array([[mimg(net.hx[v] - x0, net.Lx), mimg(net.hy[v] - y0, net.Ly)] for v in vs]), (x0, y0)


@pytest.mark.parametrize("seed", [1, 2])
def test_divisions_split_cells_exactly(seed):
    n, cap = 100, 140
    net, th, p0, v0, a0 = grown(n, seed, cap)
    rng = np.random.default_rng(seed)
    cells = rng.choice(n, 30, replace=False)
    ang = rng.uniform(0.0, np.pi, 30)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    _, _, A0, P0, _ = oracle.avm_forces(net, p0, A0=a0)
    g, th2, p02, v02, a02, made = oracle.avm_divide(net, cells, dirs, th, p0, v0, a0)
    # no cell has died: the new cells fill slots n, n+1, ... and the new vertices 2n, 2n+1, ...
    assert made.sum() == 30
    assert np.all(g.cc[n:n + 30] > 0) and np.all(g.cc[n + 30:] == 0)
    assert np.all(g.vc[3 * 2 * n:3 * (2 * n + 60)] >= 0) and np.all(g.vc[3 * (2 * n + 60):] == -1)
    check_alive_network(g, p0=p02, a0=a02)
    _, _, A1, P1, _ = oracle.avm_forces(g, p02, A0=a02)
    # divisions in order: cell k's daughter is slot n + k
    for k, c in enumerate(cells):
        d = n + k
        assert th2[d] == th2[c] and p02[d] == p0[c] and v02[d] == v0[c] and a02[d] == a0[c]
    # areas: mother = daughters; every other cell unchanged (a vertex added on a
    # straight edge does not change a polygon)
    daughters = {int(c): n + k for k, c in enumerate(cells)}
    for c in range(n):
        if c in daughters:
            continue
        assert abs(A1[c] - A0[c]) <= 1e-12
    # each division (checked against the state just before it, one at a time)
    cur, tcur, pcur, vcur, acur, ncur, vnext = net, th, p0, v0, a0, n, 2 * n  # the slots each division takes
    for k, c in enumerate(cells):
        c = int(c)
        _, _, Ab, Pb, _ = oracle.avm_forces(cur, pcur, A0=acur)
        vs, pts, (x0, y0) = polygon(cur, c)
        mean = pts.mean(0)
        nxt, tcur, pcur, vcur, acur, mk = oracle.avm_divide(cur, [c], dirs[k][None], tcur, pcur, vcur, acur)
        ncur2, vnext2 = ncur + 1, vnext + 2
        assert mk[0] == 1
        _, _, Aa, Pa, _ = oracle.avm_forces(nxt, pcur, A0=acur)
        d = ncur
        assert abs(Aa[c] + Aa[d] - Ab[c]) <= 1e-12 * Ab[c]
        A = np.array([mimg(nxt.hx[vnext] - x0, nxt.Lx), mimg(nxt.hy[vnext] - y0, nxt.Ly)])
        B = np.array([mimg(nxt.hx[vnext + 1] - x0, nxt.Lx), mimg(nxt.hy[vnext + 1] - y0, nxt.Ly)])
        chord = np.hypot(*(A - B))
        assert abs(Pa[c] + Pa[d] - (Pb[c] + 2 * chord)) <= 1e-12 * Pb[c]
        u = dirs[k]
        assert np.dot(u, A - mean) > 0 > np.dot(u, B - mean)
        # A and B lie on edges of the mother polygon
        m = len(vs)
        for X in (A, B):
            on = []
            for a in range(m):
                P, Q = pts[a], pts[(a + 1) % m]
                cross = (Q - P)[0] * (X - P)[1] - (Q - P)[1] * (X - P)[0]
                t = np.dot(X - P, Q - P) / np.dot(Q - P, Q - P)
                on.append(abs(cross) <= 1e-12 * np.dot(Q - P, Q - P) ** 0.5 and 0.0 < t < 1.0)
            assert sum(on) == 1
        cur, ncur, vnext = nxt, ncur2, vnext2
    # the step-by-step result equals the batch call
    for f in ("hx", "hy", "vc", "vn", "cc", "cv"):
        np.testing.assert_array_equal(getattr(cur, f), getattr(g, f))


def test_grown_network_keeps_stepping():
    n, cap = 100, 160
    net, th, p0, v0, a0 = grown(n, 4, cap)
    rng = np.random.default_rng(4)
    births = deaths = 0
    for k in range(300):
        if k % 50 == 0:
            alive = np.nonzero(net.cc > 0)[0]
            cells = rng.choice(alive, 8, replace=False)
            ang = rng.uniform(0.0, np.pi, 8)
            net, th, p0, v0, a0, made = oracle.avm_divide(net, cells, np.stack([np.cos(ang), np.sin(ang)], 1),
                                                          th, p0, v0, a0)
            births += int(made.sum())
        net, th, _, t2 = oracle.avm_step(net, th, p0, v0, seed=4, step=k, A0=a0, thr=0.04, t2_area=0.01, counts=True)
        deaths += t2
    assert births == 48
    # deaths free slots that later divisions take again
    assert int((net.cc > 0).sum()) == n + births - deaths
    check_alive_network(net, p0=p0, a0=a0)


def test_slots_running_out_is_an_error():
    n = 64
    net, th, p0, v0, a0 = grown(n, 5, n + 1)
    with pytest.raises(RuntimeError):
        oracle.avm_divide(net, [3, 4], [[1.0, 0.0], [0.0, 1.0]], th, p0, v0, a0)


def test_division_reuses_the_slots_a_death_freed():
    """Divisions take the lowest empty cell slot and the two lowest free vertex
    slots: after a T2 removal those are the slots it freed."""
    n, cap = 64, 80
    net, th, p0, v0, a0 = grown(n, 11, cap)
    a0[9] = 0.0
    for k in range(400):
        net, th, _, t2 = oracle.avm_step(net, th, p0, v0, seed=5, step=k, A0=a0, thr=0.04, t2_area=0.01, counts=True)
        if t2:
            break
    assert net.cc[9] == 0
    freed = sorted(np.nonzero(net.vc.reshape(-1, 3)[:2 * n, 0] < 0)[0].tolist())
    assert len(freed) == 2
    a0[9] = 1.0
    g, th2, p02, v02, a02, made = oracle.avm_divide(net, [20], [[1.0, 0.3]], th, p0, v0, a0)
    assert made[0] == 1 and g.cc[9] > 0 and np.all(g.cc[n:] == 0)
    assert all(g.vc[3 * v] >= 0 for v in freed)
    assert th2[9] == th2[20] and a02[9] == a0[20]
    check_alive_network(g, p0=p02, a0=a02)
