"""Pins the oracle of the active vertex model (AVM).

Sussman, arXiv 1702.02939: vertex forces (Eqs. A2-A5), motion (Eq. 4), T1
transitions (Fig. 1, Sec. 2.D).  Pins: the initial network is the Voronoi
tessellation (2N vertices, 3N edges, degree 3, polygons equal to the SPV
cells), forces equal finite differences of E, T1 passes keep a valid degree-3
network covering the box, the flipped edge exchanges neighbours as in Fig. 1,
and the update equals Eq. 4 written out.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def network(n, seed):
    x, y, th, L = workloads.spv_uniform(n, seed)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    return oracle.avm_build(x, y, Lx, Ly), x, y, th, Lx, Ly


def check_network(net):
    n, V = net.n, net.V
    R = oracle.MAX_RING
    assert V == 2 * n
    vc, vn = net.vc.reshape(V, 3), net.vn.reshape(V, 3)
    # every vertex has degree 3 and neighbour lists are symmetric: 3N edges
    assert set(np.bincount(net.vn, minlength=V).tolist()) == {3}
    for v in range(V):
        for s in range(3):
            w = vn[v, s]
            assert v in vn[w]
            # the edge v-w separates vc[v, s] and vc[v, s+1], which both contain w
            assert vc[v, s] in vc[w] and vc[v, (s + 1) % 3] in vc[w]
    # cell lists and vertex lists agree
    cv = net.cv.reshape(n, R)
    for c in range(n):
        m = net.cc[c]
        assert m >= 3
        for a in range(m):
            v, w = cv[c, a], cv[c, (a + 1) % m]
            assert c in vc[v]
            assert w in vn[v]  # consecutive polygon vertices are joined by an edge
    assert int(net.cc.sum()) == 3 * V  # each vertex lies on three cells
    A = oracle.avm_forces(net, 3.8)[2]
    assert np.all(A > 0)
    assert abs(A.sum() - net.Lx * net.Ly) <= 1e-10 * net.Lx * net.Ly


@pytest.mark.parametrize("n", [64, 400])
def test_voronoi_network(n):
    net, x, y, th, Lx, Ly = network(n, 5)
    check_network(net)
    A, P = oracle.avm_forces(net, 3.8)[2:4]
    topo = oracle.triangulate(x, y, Lx, Ly)
    sA, sP, _, _ = oracle.geometry(x, y, Lx, Ly, topo)
    np.testing.assert_allclose(A, sA, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(P, sP, rtol=1e-12, atol=1e-13)
    assert net.cc.sum() == 6 * n  # each vertex lies on three cells


@pytest.mark.parametrize("p0,KA,KP", [(3.8, 1.0, 1.0), (4.1, 0.5, 2.0)])
def test_vertex_forces_match_finite_differences(p0, KA, KP):
    net, *_ = network(100, 7)
    Fx, Fy, A, P, E = oracle.avm_forces(net, p0, KA=KA, KP=KP)
    scale = max(np.abs(Fx).max(), np.abs(Fy).max())
    h = 1e-6
    for v in range(0, net.V, 13):
        for arr, F in ((net.hx, Fx), (net.hy, Fy)):
            arr[v] += h
            Ep = oracle.avm_forces(net, p0, KA=KA, KP=KP)[4]
            arr[v] -= 2 * h
            Em = oracle.avm_forces(net, p0, KA=KA, KP=KP)[4]
            arr[v] += h
            assert abs(-(Ep - Em) / (2 * h) - F[v]) <= 1e-6 * scale
    # translation invariance
    assert abs(Fx.sum()) <= 1e-10 * scale * net.V and abs(Fy.sum()) <= 1e-10 * scale * net.V


@pytest.mark.parametrize("thr", [0.04, 0.1, 0.2])
def test_t1_passes_keep_a_valid_network(thr):
    net, *_ = network(400, 5)
    net2, k = oracle.avm_t1(net, thr)
    assert k > 0
    check_network(net2)
    # no edge left below the threshold unless it is a forbidden transition
    for v in range(net2.V):
        for s in range(3):
            w = net2.vn[3 * v + s]
            dx = (net2.hx[w] - net2.hx[v] + net2.Lx / 2) % net2.Lx - net2.Lx / 2
            dy = (net2.hy[w] - net2.hy[v] + net2.Ly / 2) % net2.Ly - net2.Ly / 2
            if dx * dx + dy * dy < thr * thr:
                i, kk = net2.vc[3 * v + s], net2.vc[3 * v + (s + 1) % 3]
                assert net2.cc[i] <= 3 or net2.cc[kk] <= 3


def adjacent(net, a, b):
    """Cells a and b share an edge (two consecutive vertices)."""
    R = oracle.MAX_RING
    va = set(net.cv[a * R:a * R + net.cc[a]].tolist())
    vb = set(net.cv[b * R:b * R + net.cc[b]].tolist())
    return len(va & vb) >= 2


def test_t1_exchanges_neighbours_as_in_figure_1():
    net, *_ = network(400, 5)
    # shortest edge
    best = None
    for v in range(net.V):
        for s in range(3):
            w = net.vn[3 * v + s]
            if w <= v:
                continue
            dx = (net.hx[w] - net.hx[v] + net.Lx / 2) % net.Lx - net.Lx / 2
            dy = (net.hy[w] - net.hy[v] + net.Ly / 2) % net.Ly - net.Ly / 2
            d = math.hypot(dx, dy)
            if best is None or d < best[0]:
                best = (d, v, s, w, dx, dy)
    d, v, s, w, ex, ey = best
    i, k, j = net.vc[3 * v + s], net.vc[3 * v + (s + 1) % 3], net.vc[3 * v + (s + 2) % 3]
    l = [c for c in net.vc[3 * w:3 * w + 3] if c not in (i, k)][0]
    assert adjacent(net, i, k) and not adjacent(net, j, l)
    thr = d * 1.0001  # only this edge qualifies
    net2, nt1 = oracle.avm_t1(net, thr)
    assert nt1 == 1
    assert adjacent(net2, j, l) and not adjacent(net2, i, k)
    # the new edge: length 1.5 thr, perpendicular to the old one, same midpoint
    fx = (net2.hx[w] - net2.hx[v] + net2.Lx / 2) % net2.Lx - net2.Lx / 2
    fy = (net2.hy[w] - net2.hy[v] + net2.Ly / 2) % net2.Ly - net2.Ly / 2
    assert abs(math.hypot(fx, fy) - 1.5 * thr) < 1e-12
    assert abs(fx * ex + fy * ey) < 1e-12
    mx0 = net.hx[v] + ex / 2
    mx1 = net2.hx[v] + fx / 2
    assert abs((mx1 - mx0 + net.Lx / 2) % net.Lx - net.Lx / 2) < 1e-12
    check_network(net2)


def test_one_transition_per_cell_per_pass():
    """Two candidate edges of one cell: the first pass applies only the one
    with the smaller edge id; the other follows in a later pass."""
    net, *_ = network(400, 5)
    R = oracle.MAX_RING
    c = int(np.argmax(net.cc))  # a cell with many edges
    verts = net.cv[c * R:c * R + net.cc[c]]
    # make two non-adjacent edges of c short by moving vertex pairs together
    e1 = (verts[0], verts[1])
    e2 = (verts[3], verts[4])
    for (a, b) in (e1, e2):
        dx = (net.hx[b] - net.hx[a] + net.Lx / 2) % net.Lx - net.Lx / 2
        dy = (net.hy[b] - net.hy[a] + net.Ly / 2) % net.Ly - net.Ly / 2
        net.hx[b] = (net.hx[a] + 0.01 * dx + net.Lx) % net.Lx
        net.hy[b] = (net.hy[a] + 0.01 * dy + net.Ly) % net.Ly
    one, n1 = oracle.avm_t1(net, 0.03, cap=1, allow_cap=True)
    assert n1 >= 1
    full, nf = oracle.avm_t1(net, 0.03)
    assert nf >= n1 + 1
    check_network(full)


def test_step_formula_without_forces():
    """K_A = K_P = 0: each vertex moves by dt (v0/3) sum of its cells' directors
    (Eq. 4), then the directors rotate by sqrt(2 D_r dt) xi."""
    net, x, y, th, Lx, Ly = network(200, 9)
    v0, dt = 0.3, 0.01
    net2, th2, nt = oracle.avm_step(net, th, 3.8, v0, seed=3, step=7, KA=0.0, KP=0.0, dt=dt, thr=0.0)
    vc = net.vc.reshape(-1, 3)
    ex = net.hx + dt * v0 / 3.0 * np.cos(th[vc]).sum(1)
    ey = net.hy + dt * v0 / 3.0 * np.sin(th[vc]).sum(1)
    assert np.abs((net2.hx - ex + Lx / 2) % Lx - Lx / 2).max() < 1e-12
    assert np.abs((net2.hy - ey + Ly / 2) % Ly - Ly / 2).max() < 1e-12
    xi = np.array([oracle.director_noise(3, c, 7) for c in range(200)])
    np.testing.assert_allclose(th2, th + math.sqrt(2 * dt) * xi, rtol=0, atol=1e-14)


def test_gradient_descent_lowers_energy():
    net, x, y, th, Lx, Ly = network(200, 4)
    E = [oracle.avm_forces(net, 3.7)[4]]
    for step in range(6):
        net, th, _ = oracle.avm_step(net, th, 3.7, 0.0, seed=1, step=step, Dr=0.0, dt=0.005, thr=0.0)
        E.append(oracle.avm_forces(net, 3.7)[4])
    assert all(b < a for a, b in zip(E, E[1:]))
