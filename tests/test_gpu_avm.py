"""GPU active vertex model (AVM) against the oracle.

Sussman, arXiv 1702.02939, Sec. 2.D: vertex forces (Eqs. A2-A5), motion
(Eq. 4), T1 transitions (Fig. 1).  The network built from the seeds, the T1
decisions and every list of the network must be bit-exact; forces within
1e-10 max|F|; positions within 1e-12 L per step.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1702_02939_gb300 as cg  # noqa: E402

F_TOL = 1e-10
X_TOL = 1e-12
R = oracle.MAX_RING


def seeds(n, iseed, L=None):
    x, y, th, Lr = workloads.spv_uniform(n, iseed, L)
    Lx, Ly, q = oracle.box(Lr)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    return xs, ys, th, Lr, Lx, Ly


def make(n, iseed, L=None, **kw):
    xs, ys, th, Lr, Lx, Ly = seeds(n, iseed, L)
    sim = cg.AVM(n, Lr, Lr, xs, ys, th, **kw)
    return sim, xs, ys, th, Lx, Ly


def wrapdiff(a, b, L):
    return (a - b + L / 2) % L - L / 2


def gpu_net(sim, Lx, Ly):
    hx, hy, th = (t.cpu().numpy() for t in sim.state())
    vc, vn, cc, cv = (t.cpu().numpy() for t in sim.topology())
    return oracle.AvmNet(sim.n, Lx, Ly, hx, hy, vc.reshape(-1), vn.reshape(-1), cc, cv.reshape(-1)), th


def assert_same_network(g, o, tol=X_TOL):
    np.testing.assert_array_equal(g.vc, o.vc)
    np.testing.assert_array_equal(g.vn, o.vn)
    np.testing.assert_array_equal(g.cc, o.cc)
    np.testing.assert_array_equal(g.cv, o.cv)
    assert np.abs(wrapdiff(g.hx, o.hx, o.Lx)).max() <= tol * o.Lx
    assert np.abs(wrapdiff(g.hy, o.hy, o.Ly)).max() <= tol * o.Ly


def load(sim, net, theta=None):
    sim.set_state(net.hx, net.hy, theta, net.vc, net.vn, net.cc, net.cv)


def test_smallest_box_is_refused_cleanly():
    """16 cells at unit density (L = 4): a Voronoi cell can be wider than the
    cell-list search of the seed triangulation covers in so small a box; the
    library reports CG_EBOX_TOO_SMALL instead of a wrong network."""
    with pytest.raises(cg.CellgbError) as e:
        make(16, 1)
    assert e.value.code == -7


@pytest.mark.parametrize("n,iseed", [(64, 2), (400, 3), (4096, 4)])
def test_network_build_matches_oracle(n, iseed):
    sim, xs, ys, th, Lx, Ly = make(n, iseed)
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, oracle.avm_build(xs, ys, Lx, Ly))
    np.testing.assert_array_equal(gth, th)
    sim.close()


@pytest.mark.parametrize("p0,KA,KP", [(3.8, 1.0, 1.0), (4.1, 0.5, 2.0)])
def test_forces_match_oracle(p0, KA, KP):
    n = 1000
    sim, xs, ys, th, Lx, Ly = make(n, 5, p0=p0, KA=KA, KP=KP)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    load(sim, net)  # identical positions on both sides
    Fx, Fy, E = sim.forces()
    A, P = (t.cpu().numpy() for t in sim.geometry())
    oFx, oFy, oA, oP, oE = oracle.avm_forces(net, p0, KA=KA, KP=KP)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    assert np.abs(Fy.cpu().numpy() - oFy).max() <= F_TOL * scale
    np.testing.assert_allclose(A, oA, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(P, oP, rtol=1e-12, atol=1e-13)
    assert abs(E - oE) <= 1e-11 * abs(oE)
    sim.close()


def test_per_cell_p0_and_v0():
    n = 400
    sim, xs, ys, th, Lx, Ly = make(n, 6, t1_threshold=0.0)
    rng = np.random.default_rng(2)
    p0 = rng.uniform(3.6, 4.0, n)
    v0 = rng.uniform(0.0, 0.3, n)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    load(sim, net, th)
    sim.set_p0(p0)
    sim.set_v0(v0)
    Fx, Fy, _ = sim.forces()
    oFx, oFy, *_ = oracle.avm_forces(net, p0)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    sim.step(1)
    g, gth = gpu_net(sim, Lx, Ly)
    o, oth, _ = oracle.avm_step(net, th, p0, v0, seed=0, step=0, thr=0.0)
    assert_same_network(g, o)
    np.testing.assert_allclose(gth, oth, rtol=0, atol=1e-13)
    sim.close()


@pytest.mark.parametrize("thr", [0.04, 0.1, 0.2])
def test_t1_passes_match_oracle(thr):
    """Same network on both sides, then T1 passes only: the winners of every
    pass (smallest edge id on each of the four cells) and the rewired lists
    must agree exactly; thr = 0.2 gives many conflicting candidates.  The
    fresh network has 171, 469 and 929 edges below the three thresholds, so
    the first pass is applied by every block of the apply kernel and the
    later, smaller passes by its first block alone."""
    n = 2000
    sim, xs, ys, th, Lx, Ly = make(n, 7, t1_threshold=thr)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    o, k = oracle.avm_t1(net, thr)
    assert k > 0
    load(sim, net)
    sim.t1()
    g, _ = gpu_net(sim, Lx, Ly)
    assert_same_network(g, o)
    c = sim.counters()
    assert c["t1_total"] == k and c["status"] == 0
    sim.close()


def edge_lengths(net):
    """(v, w, |h_w - h_v|) for every edge v < w, the squared length rounded as
    the T1 rule states (each product and the sum on its own)."""
    vn = net.vn.reshape(-1, 3)
    out = []
    for v in range(net.V):
        for s in range(3):
            w = int(vn[v, s])
            if w <= v:
                continue
            dx = (net.hx[w] - net.hx[v] + net.Lx / 2) % net.Lx - net.Lx / 2
            dy = (net.hy[w] - net.hy[v] + net.Ly / 2) % net.Ly - net.Ly / 2
            out.append((v, w, np.sqrt(dx * dx + dy * dy)))
    return out


@pytest.mark.parametrize("side", [-1, +1])
def test_t1_threshold_at_an_edge_length(side):
    """Thresholds one ulp either side of existing edge lengths put those edges
    inside the band where the FP32 length filter defers to FP64: the decisions
    and the resulting networks must still equal the oracle's."""
    n = 2000
    xs, ys, th, Lr, Lx, Ly = seeds(n, 14)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    lengths = sorted(l for _, _, l in edge_lengths(net) if 0.05 < l < 0.12)
    for l in lengths[:: max(1, len(lengths) // 3)][:3]:
        thr = float(np.nextafter(l, np.inf if side > 0 else 0.0))
        sim = cg.AVM(n, Lr, Lr, xs, ys, th, t1_threshold=thr)
        load(sim, net)
        o, k = oracle.avm_t1(net, thr)
        sim.t1()
        g, _ = gpu_net(sim, Lx, Ly)
        assert_same_network(g, o)
        assert sim.counters()["t1_total"] == k
        sim.close()


def test_t1_cap_status():
    """Candidates left after t1_cap passes raise the T1-cap status on the host."""
    n = 2000
    sim, xs, ys, th, Lx, Ly = make(n, 7, t1_threshold=0.3, t1_cap=1)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    with pytest.raises(oracle.OracleError):
        oracle.avm_t1(net, 0.3, cap=1)  # the oracle reports the same situation
    load(sim, net)
    with pytest.raises(cg.CellgbError) as e:
        sim.t1()
    assert e.value.code == -10
    sim.close()


@pytest.mark.parametrize("n,iseed,thr,steps", [(400, 8, 0.04, 1), (2000, 9, 0.1, 1), (2000, 10, 0.1, 5)])
def test_steps_match_oracle(n, iseed, thr, steps):
    p0, v0, dt = 3.8, 0.1, 0.01
    sim, xs, ys, th, Lx, Ly = make(n, iseed, p0=p0, v0=v0, dt=dt, t1_threshold=thr, seed=11)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    load(sim, net, th)
    sim.step(steps)
    g, gth = gpu_net(sim, Lx, Ly)
    o, oth, total = net, th, 0
    for s in range(steps):
        o, oth, k = oracle.avm_step(o, oth, p0, v0, seed=11, step=s, dt=dt, thr=thr)
        total += k
    assert total > 0
    assert_same_network(g, o, tol=X_TOL * steps)
    np.testing.assert_allclose(gth, oth, rtol=0, atol=1e-13 * steps)
    c = sim.counters()
    assert c["steps"] == steps and c["t1_total"] == total
    sim.close()


def test_profiled_steps_equal_graph_steps():
    """The eagerly launched, host-controlled steps of the profiler advance the
    state bit-identically to the graph steps with the conditional T1 loop."""
    n = 2000
    a, xs, ys, th, Lx, Ly = make(n, 13, t1_threshold=0.1, seed=5)
    b, *_ = make(n, 13, t1_threshold=0.1, seed=5)
    a.step(6)
    ph = b.profile(6)
    assert ph["t1_passes"] >= 6
    ga, tha = gpu_net(a, Lx, Ly)
    gb, thb = gpu_net(b, Lx, Ly)
    for f in ("hx", "hy", "vc", "vn", "cc", "cv"):
        np.testing.assert_array_equal(getattr(ga, f), getattr(gb, f))
    np.testing.assert_array_equal(tha, thb)
    assert a.counters() == b.counters()
    a.close()
    b.close()


def check_network_valid(sim, Lx, Ly, p0):
    """Properties that hold at any size: degree 3, symmetric neighbour lists,
    cell lists consistent with vertex lists, areas positive and tiling the box;
    vertices freed and cells emptied by T2s (vc, vn = -1; cc = 0, A = 0) excluded,
    two vertices per remaining cell."""
    g, _ = gpu_net(sim, Lx, Ly)
    V, n = g.V, g.n
    vc, vn = g.vc.reshape(V, 3), g.vn.reshape(V, 3)
    free = vc[:, 0] < 0
    assert np.all(vc[free] == -1) and np.all(vn[free] == -1)
    alive = g.cc > 0
    assert int((~free).sum()) == 2 * int(alive.sum())
    live = np.nonzero(~free)[0]
    assert np.all(np.bincount(vn[live].ravel(), minlength=V)[live] == 3)
    for s in range(3):
        w = vn[live, s]
        assert np.all(w >= 0) and not np.any(free[w])
        assert np.all((vn[w] == live[:, None]).any(1))
        assert np.all(alive[vc[live, s]])
    assert int(g.cc.sum()) == 3 * len(live)
    cv = g.cv.reshape(n, R)
    for c in range(0, n, max(1, n // 300)):
        for a in range(g.cc[c]):
            assert c in vc[cv[c, a]]
    A, P = (t.cpu().numpy() for t in sim.geometry())
    assert np.all(A[alive] > 0) and np.all(A[~alive] == 0.0)
    assert abs(A.sum() - Lx * Ly) <= 1e-9 * Lx * Ly
    return g


def test_long_run_keeps_a_valid_network():
    n = 4096
    sim, xs, ys, th, Lx, Ly = make(n, 12, p0=3.8, v0=0.1, t1_threshold=0.04, seed=3)
    sim.step(300)
    sim.sync()
    check_network_valid(sim, Lx, Ly, 3.8)
    assert sim.counters()["t1_total"] > 0
    sim.close()


def test_full_size_workload():
    """N = 65536, L = 256 (the benchmark workload): network build bit-exact,
    forces within tolerance, one step (move, directors, T1) exact, then 50
    more steps keep a valid network."""
    n, p0, v0, thr = 65536, 3.8, 0.1, 0.04
    sim, xs, ys, th, Lx, Ly = make(n, 1, p0=p0, v0=v0, t1_threshold=thr, seed=1)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    g, _ = gpu_net(sim, Lx, Ly)
    assert_same_network(g, net)
    load(sim, net, th)
    Fx, Fy, _ = sim.forces()
    oFx, oFy, *_ = oracle.avm_forces(net, p0)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    sim.step(1)
    g, gth = gpu_net(sim, Lx, Ly)
    o, oth, k = oracle.avm_step(net, th, p0, v0, seed=1, step=0, thr=thr)
    assert k > 0
    assert_same_network(g, o)
    sim.step(50)
    check_network_valid(sim, Lx, Ly, p0)
    sim.close()


def test_long_run_ensemble_statistics_match_oracle():
    """Long AVM runs (N = 400, p0 = 3.8, v0 = 0.1, T1 threshold 0.04, 1000
    steps, eight seeds): the ensemble mean shape index agrees within 1% and
    the vertex mean-squared displacement within its seed-to-seed standard
    error."""
    n, K, p0, v0, thr = 400, 1000, 3.8, 0.1, 0.04
    qg, qo, mg, mo = [], [], [], []
    for s in range(8):
        sim, xs, ys, th, Lx, Ly = make(n, 200 + s, p0=p0, v0=v0, t1_threshold=thr, seed=s)
        net = oracle.avm_build(xs, ys, Lx, Ly)
        load(sim, net, th)
        sim.step(K)
        g, _ = gpu_net(sim, Lx, Ly)
        A, P = (t.cpu().numpy() for t in sim.geometry())
        sim.close()
        o, oth = net, th
        for k in range(K):
            o, oth, _ = oracle.avm_step(o, oth, p0, v0, seed=s, step=k, thr=thr)
        _, _, oA, oP, _ = oracle.avm_forces(o, p0)
        qg.append((P / np.sqrt(A)).mean())
        qo.append((oP / np.sqrt(oA)).mean())
        mg.append((wrapdiff(g.hx, net.hx, Lx) ** 2 + wrapdiff(g.hy, net.hy, Ly) ** 2).mean())
        mo.append((wrapdiff(o.hx, net.hx, Lx) ** 2 + wrapdiff(o.hy, net.hy, Ly) ** 2).mean())
    qg, qo, mg, mo = (np.asarray(v) for v in (qg, qo, mg, mo))
    se = max(mg.std(ddof=1), mo.std(ddof=1)) / np.sqrt(len(mg))
    print(f"q: gpu {qg.mean():.6f} oracle {qo.mean():.6f}; MSD: gpu {mg.mean():.6f} oracle {mo.mean():.6f} se {se:.2e}")
    assert abs(qg.mean() - qo.mean()) <= 0.01 * qo.mean()
    assert abs(mg.mean() - mo.mean()) <= se


def test_corrupted_network_is_refused():
    """A network handed in with an out-of-range neighbour or a non-finite
    position is refused with CG_EINVAL before any step uses it."""
    n = 400
    sim, xs, ys, th, Lx, Ly = make(n, 15)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    vn = net.vn.copy()
    vn[10] = 10 * net.V
    with pytest.raises(cg.CellgbError) as e:
        sim.set_state(net.hx, net.hy, th, net.vc, vn, net.cc, net.cv)
    assert e.value.code == -1
    with pytest.raises(cg.CellgbError):
        sim.step(1)  # the context keeps the error: no step runs on it
    sim.close()
    sim, *_ = make(n, 15)
    hx = net.hx.copy()
    hx[3] = float("nan")
    with pytest.raises(cg.CellgbError) as e:
        sim.set_state(hx, net.hy, th, net.vc, net.vn, net.cc, net.cv)
    assert e.value.code == -1
    sim.close()


def test_rectangular_box():
    """AVM in a 40 x 10 box: network build and one step equal the oracle."""
    n, Lxr, Lyr = 400, 40.0, 10.0
    x, y, th = workloads.spv_uniform_rect(n, 16, Lxr, Lyr)
    Lx, Ly, q = oracle.box(Lxr, Lyr)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    sim = cg.AVM(n, Lxr, Lyr, xs, ys, th, t1_threshold=0.1, seed=3)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    g, _ = gpu_net(sim, Lx, Ly)
    assert_same_network(g, net)
    load(sim, net, th)
    sim.step(1)
    g, gth = gpu_net(sim, Lx, Ly)
    o, oth, _ = oracle.avm_step(net, th, 3.8, 0.1, seed=3, step=0, thr=0.1)
    assert_same_network(g, o)
    sim.close()


def test_t2_dying_cells_match_oracle():
    """Cells given A0 = 0 shrink, become triangles through T1s and are removed
    by T2s: every step (move, directors, T1 and T2 passes) equals the oracle's
    step from the same state (network exact, positions within 1e-12 L)."""
    n, p0, v0, thr, t2 = 400, 3.8, 0.05, 0.04, 0.01
    sim, xs, ys, th, Lx, Ly = make(n, 21, p0=p0, v0=v0, t1_threshold=thr, t2_area=t2, seed=4)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    rng = np.random.default_rng(1)
    a0 = np.ones(n)
    dying = rng.choice(n, 8, replace=False)
    a0[dying] = 0.0
    sim.set_a0(a0)
    load(sim, net, th)
    o, oth = net, th
    total_t1 = total_t2 = 0
    for k in range(160):
        sim.step(1)
        g, gth = gpu_net(sim, Lx, Ly)
        o, oth, k1, k2 = oracle.avm_step(o, oth, p0, v0, seed=4, step=k, A0=a0, thr=thr, t2_area=t2, counts=True)
        assert_same_network(g, o)
        np.testing.assert_allclose(gth, oth, rtol=0, atol=1e-13)
        total_t1 += k1
        total_t2 += k2
        load(sim, o, oth)  # the next step from the oracle's state
    assert total_t2 >= 4
    assert set(np.nonzero(o.cc == 0)[0].tolist()) <= set(dying.tolist())
    c = sim.counters()
    assert c["t2_total"] == total_t2 and c["t1_total"] == total_t1
    Fx, Fy, _ = sim.forces()
    oFx, oFy, *_ = oracle.avm_forces(o, p0, A0=a0)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    sim.close()


def test_per_cell_a0_is_checked():
    sim, *_ = make(400, 22)
    bad = np.ones(400)
    bad[3] = -1.0
    with pytest.raises(cg.CellgbError) as e:
        sim.set_a0(bad)
    assert e.value.code == -1
    sim.close()


def test_full_size_with_cell_death():
    """N = 65536 with 1% of the cells set to die: after 400 graph steps every
    dying cell that was removed is one of them, the counters agree with the
    emptied cells, and the network is still a valid tiling."""
    n, p0, v0, thr = 65536, 3.8, 0.1, 0.04
    sim, xs, ys, th, Lx, Ly = make(n, 1, p0=p0, v0=v0, t1_threshold=thr, t2_area=0.01, seed=1)
    rng = np.random.default_rng(7)
    a0 = np.ones(n)
    dying = rng.choice(n, n // 100, replace=False)
    a0[dying] = 0.0
    sim.set_a0(a0)
    sim.step(400)
    sim.sync()
    g = check_network_valid(sim, Lx, Ly, p0)
    removed = set(np.nonzero(g.cc == 0)[0].tolist())
    assert len(removed) > n // 200 and removed <= set(dying.tolist())
    assert sim.counters()["t2_total"] == len(removed)
    sim.close()


def test_divisions_match_oracle():
    """Divisions along given directions give the oracle's network (topology
    exact, new vertex positions within 1e-12 L), and the grown network then
    steps like the oracle's (T1 and T2 passes, new cells' directors)."""
    n, cap, p0, v0, thr = 100, 150, 3.8, 0.05, 0.04
    sim, xs, ys, th, Lx, Ly = make(n, 31, p0=p0, v0=v0, t1_threshold=thr, t2_area=0.01, seed=6, capacity=cap)
    assert sim.n == cap and sim.V == 2 * cap
    net = oracle.avm_build(xs, ys, Lx, Ly).with_capacity(cap)
    theta = np.concatenate([th, np.zeros(cap - n)])
    pa, va, aa = np.full(cap, p0), np.full(cap, v0), np.ones(cap)
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, net)
    rng = np.random.default_rng(3)
    cells = rng.choice(n, 30, replace=False)
    ang = rng.uniform(0.0, np.pi, 30)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    made = sim.divide(cells, dirs)
    o, theta, pa, va, aa, omade = oracle.avm_divide(net, cells, dirs, theta, pa, va, aa)
    np.testing.assert_array_equal(made, omade)
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, o)
    np.testing.assert_array_equal(gth, theta)
    # a few of the new cells die
    aa[n:n + 3] = 0.0
    sim.set_a0(aa)
    for k in range(120):
        sim.step(1)
        g, gth = gpu_net(sim, Lx, Ly)
        o, theta, _, _ = oracle.avm_step(o, theta, pa, va, seed=6, step=k, A0=aa, thr=thr, t2_area=0.01, counts=True)
        assert_same_network(g, o)
        np.testing.assert_allclose(gth, theta, rtol=0, atol=1e-13)
        load(sim, o, theta)
    check_network_valid(sim, Lx, Ly, p0)
    assert int((g.cc == 0).sum()) >= 1
    sim.close()


def test_divisions_in_conflict_match_oracle():
    """Divisions that touch one another within one call -- the same cell
    twice, neighbouring cells, the empty slot an earlier division of the call
    fills -- give the network of doing them one after the other, as the
    oracle does; and a large call (many cells, few conflicts) as well."""
    n, cap, p0, v0 = 400, 520, 3.8, 0.05
    sim, xs, ys, th, Lx, Ly = make(n, 35, p0=p0, v0=v0, t1_threshold=0.04, seed=9, capacity=cap)
    net = oracle.avm_build(xs, ys, Lx, Ly).with_capacity(cap)
    theta = np.concatenate([th, np.zeros(cap - n)])
    pa, va, aa = np.full(cap, p0), np.full(cap, v0), np.ones(cap)
    g, _ = gpu_net(sim, Lx, Ly)
    v7 = int(g.cv[7 * R])  # a vertex of cell 7; its other cells are neighbours of 7
    nb7 = [int(c) for c in g.vc[3 * v7:3 * v7 + 3] if c != 7][0]
    cells = np.array([7, 7, nb7, n, 7, n, 11, 12, 13, 14, 200, 201, n + 1])
    rng = np.random.default_rng(4)
    ang = rng.uniform(0.0, np.pi, len(cells))
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    made = sim.divide(cells, dirs)
    o, theta, pa, va, aa, omade = oracle.avm_divide(net, cells, dirs, theta, pa, va, aa)
    np.testing.assert_array_equal(made, omade)
    assert made[3] == 1  # slot n, filled by the first division, was divided in the same call
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, o)
    np.testing.assert_array_equal(gth, theta)
    live = np.nonzero(o.cc > 0)[0]
    cells = rng.choice(live, 100, replace=False)
    ang = rng.uniform(0.0, np.pi, 100)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    made = sim.divide(cells, dirs)
    o, theta, pa, va, aa, omade = oracle.avm_divide(o, cells, dirs, theta, pa, va, aa)
    np.testing.assert_array_equal(made, omade)
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, o)
    check_network_valid(sim, Lx, Ly, p0)
    sim.close()


def test_divisions_beyond_one_window_match_oracle():
    """A call with more divisions than one round's window (1024), some of them
    on neighbouring cells, on a re-sorted storage: the network of doing them
    one after the other, as the oracle does."""
    n, cap, p0, v0 = 4096, 5400, 3.8, 0.05
    sim, xs, ys, th, Lx, Ly = make(n, 36, p0=p0, v0=v0, t1_threshold=0.04, seed=10, capacity=cap, sort_every=50)
    net = oracle.avm_build(xs, ys, Lx, Ly).with_capacity(cap)
    theta = np.concatenate([th, np.zeros(cap - n)])
    pa, va, aa = np.full(cap, p0), np.full(cap, v0), np.ones(cap)
    rng = np.random.default_rng(7)
    cells = rng.choice(n, 1200, replace=False)
    ang = rng.uniform(0.0, np.pi, cells.size)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    made = sim.divide(cells, dirs)
    o, theta, pa, va, aa, omade = oracle.avm_divide(net, cells, dirs, theta, pa, va, aa)
    np.testing.assert_array_equal(made, omade)
    assert made.sum() > 1100
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, o)
    np.testing.assert_array_equal(gth, theta)
    check_network_valid(sim, Lx, Ly, p0)
    sim.close()


def test_division_slots_are_checked():
    n = 64
    sim, *_ = make(n, 32, capacity=n + 1)
    with pytest.raises(cg.CellgbError) as e:
        sim.divide([3, 4], [[1.0, 0.0], [0.0, 1.0]])
    assert e.value.code == -1
    assert sim.divide([3], [[1.0, 0.0]])[0] == 1
    with pytest.raises(cg.CellgbError):
        sim.divide([5], [[0.0, 1.0]])
    sim.close()


def test_full_size_growth():
    """N = 65536 seeds with room for 4096 more cells: 4000 divisions, then 200
    graph steps with T1 and T2 passes keep a valid tiling, one cell per
    division made and none but those the T2s removed."""
    n, cap = 65536, 65536 + 4096
    sim, xs, ys, th, Lx, Ly = make(n, 1, p0=3.8, v0=0.1, t1_threshold=0.04, t2_area=0.01, seed=1, capacity=cap)
    rng = np.random.default_rng(9)
    cells = rng.choice(n, 4000, replace=False)
    ang = rng.uniform(0.0, np.pi, 4000)
    made = sim.divide(cells, np.stack([np.cos(ang), np.sin(ang)], 1))
    assert made.sum() >= 3990
    sim.step(200)
    sim.sync()
    g = check_network_valid(sim, Lx, Ly, 3.8)
    # a daughter that is a small triangle may be removed by a T2 meanwhile
    assert int((g.cc > 0).sum()) == n + int(made.sum()) - sim.counters()["t2_total"]
    sim.close()


def test_full_size_five_thousand_steps():
    """The AVM workload's length: N = 65536, 5000 graph steps with T1 passes;
    the network is still a valid tiling and the T1 count is in line with the
    per-step rate of the benchmark (about 16 per step)."""
    n = 65536
    sim, xs, ys, th, Lx, Ly = make(n, 1, p0=3.8, v0=0.1, t1_threshold=0.04, seed=1)
    sim.step(5000)
    sim.sync()
    check_network_valid(sim, Lx, Ly, 3.8)
    c = sim.counters()
    assert c["steps"] == 5000 and 5 * 5000 < c["t1_total"] < 50 * 5000
    sim.close()


def test_resume_after_deaths_and_divisions_is_bit_identical():
    """A run with dying cells and divisions, saved (positions, directors,
    network, step counter) and resumed in a fresh context, continues bit for
    bit like the original (divisions take the same slots)."""
    n, cap = 400, 440
    kw = dict(p0=3.8, v0=0.1, t1_threshold=0.04, t2_area=0.01, seed=12, capacity=cap)
    a, xs, ys, th, Lx, Ly = make(n, 41, **kw)
    a0 = np.ones(cap)
    rng = np.random.default_rng(4)
    dying = rng.choice(n, 6, replace=False)
    a0[dying] = 0.0
    a.set_a0(a0)
    live = np.setdiff1d(np.arange(n), dying)
    c1, c2 = rng.choice(live, 8, replace=False), rng.choice(live, 8, replace=False)
    d1, d2 = rng.normal(size=(8, 2)), rng.normal(size=(8, 2))
    a.step(60)
    a.divide(c1, d1)
    a.step(20)
    hx, hy, theta = (t.clone() for t in a.state())
    topo = [t.clone() for t in a.topology()]
    p0s, v0s, a0s = a.cell_params()  # divisions may have put new cells in emptied slots
    step = a.counters()["steps"]
    a.divide(c2, d2)
    a.step(40)
    b, *_ = make(n, 42, **kw)  # other seeds: everything comes from the saved state
    b.set_p0(p0s)
    b.set_v0(v0s)
    b.set_a0(a0s)
    b.set_state(hx, hy, theta, *topo)
    b.set_step(step)
    b.divide(c2, d2)
    b.step(40)
    for ta, tb in zip(a.state(), b.state()):
        assert torch.equal(ta, tb)
    for ta, tb in zip(a.topology(), b.topology()):
        assert torch.equal(ta, tb)
    assert a.counters()["t2_total"] > 0
    a.close()
    b.close()


def test_divisions_after_deaths_match_oracle():
    """Dying cells removed by T2s free their slots; later divisions take the
    lowest empty and free slots, as in the oracle."""
    n, cap, p0, v0, thr = 100, 120, 3.8, 0.05, 0.04
    sim, xs, ys, th, Lx, Ly = make(n, 33, p0=p0, v0=v0, t1_threshold=thr, t2_area=0.01, seed=8, capacity=cap)
    net = oracle.avm_build(xs, ys, Lx, Ly).with_capacity(cap)
    theta = np.concatenate([th, np.zeros(cap - n)])
    pa, va, aa = np.full(cap, p0), np.full(cap, v0), np.ones(cap)
    rng = np.random.default_rng(2)
    dying = rng.choice(n, 4, replace=False)
    aa[dying] = 0.0
    sim.set_a0(aa)
    o = net
    for k in range(150):
        sim.step(1)
        o, theta, _, _ = oracle.avm_step(o, theta, pa, va, seed=8, step=k, A0=aa, thr=thr, t2_area=0.01, counts=True)
        g, gth = gpu_net(sim, Lx, Ly)
        assert_same_network(g, o)
        load(sim, o, theta)
    removed = np.nonzero(o.cc[:n] == 0)[0]
    assert len(removed) >= 2
    live = np.nonzero(o.cc > 0)[0]
    cells = rng.choice(live, 10, replace=False)
    dirs = rng.normal(size=(10, 2))
    made = sim.divide(cells, dirs)
    o, theta, pa, va, aa, omade = oracle.avm_divide(o, cells, dirs, theta, pa, va, aa)
    np.testing.assert_array_equal(made, omade)
    g, gth = gpu_net(sim, Lx, Ly)
    assert_same_network(g, o)
    assert np.all(o.cc[removed] > 0)  # the emptied slots are taken first
    sim.close()
