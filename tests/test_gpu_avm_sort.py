"""Storage order of the AVM: Hilbert re-sort of the vertex and cell slots.

Sussman, arXiv 1702.02939, Sec. 2.B: the arrays are re-sorted so that
particles close in space sit close in memory.  Every id of the API is a tag
fixed when a vertex or cell comes into being, and every id-dependent rule
(T1 and T2 priorities, the end a T1 edge is taken from, the vertex a T2
keeps, the noise counter, the slots divisions fill) uses the tags, so a run
that re-sorts gives bit for bit the results of one that never does: the same
positions, directors, network, forces, energy, per-cell parameters and
counters, through T1s, T2s (cell death) and divisions.
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


def seeds(n, iseed):
    x, y, th, Lr = workloads.spv_uniform(n, iseed)
    Lx, Ly, q = oracle.box(Lr)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    return xs, ys, th, Lr, Lx, Ly


def outputs(sim):
    """Everything the API reports, as host arrays."""
    out = [t.cpu().numpy() for t in sim.state()]
    out += [t.cpu().numpy() for t in sim.topology()]
    out += [t.cpu().numpy() for t in sim.geometry()]
    Fx, Fy, E = sim.forces()
    out += [Fx.cpu().numpy(), Fy.cpu().numpy(), np.array([E])]
    out += [t.cpu().numpy() for t in sim.cell_params()]
    return out


def assert_identical(a, b):
    for x, y in zip(outputs(a), outputs(b)):
        assert x.dtype == y.dtype and x.shape == y.shape
        np.testing.assert_array_equal(x, y)
    assert a.counters() == b.counters()


def assert_permutation(tags, moved):
    t = tags.cpu().numpy()
    np.testing.assert_array_equal(np.sort(t), np.arange(t.size))
    assert (t != np.arange(t.size)).any() == moved


def test_resort_keeps_every_result_through_deaths_and_divisions():
    n, cap = 4096, 4400
    xs, ys, th, Lr, Lx, Ly = seeds(n, 51)
    kw = dict(p0=3.8, v0=0.1, t1_threshold=0.06, t2_area=0.01, seed=9, capacity=cap)
    a = cg.AVM(n, Lr, Lr, xs, ys, th, **kw)
    b = cg.AVM(n, Lr, Lr, xs, ys, th, sort_every=7, **kw)
    va, ca = a.storage_tags()
    vb, cb = b.storage_tags()
    assert_permutation(va, False)
    assert_permutation(ca, False)
    assert_permutation(vb, True)  # sorted at creation
    assert_permutation(cb, True)
    assert_identical(a, b)
    rng = np.random.default_rng(5)
    a0 = np.ones(cap)
    dying = rng.choice(n, 40, replace=False)
    a0[dying] = 0.0
    p0 = np.full(cap, 3.8)
    p0[rng.choice(n, 100, replace=False)] = 3.95
    for s in (a, b):
        s.set_a0(a0)
        s.set_p0(p0)
    a.step(80)
    b.step(80)
    assert_identical(a, b)
    assert a.counters()["t2_total"] > 0 and a.counters()["t1_total"] > 0
    live = np.nonzero(a.topology()[2].cpu().numpy() > 0)[0]
    cells = rng.choice(live, 60, replace=False)
    dirs = rng.normal(size=(60, 2))
    np.testing.assert_array_equal(a.divide(cells, dirs), b.divide(cells, dirs))
    assert_identical(a, b)
    v0 = np.full(cap, 0.1)
    v0[cells] = 0.2
    for s in (a, b):
        s.set_v0(v0)
    a.step(60)
    b.step(60)
    b.sort()  # an explicit re-sort between steps changes nothing either
    assert_identical(a, b)
    a.close()
    b.close()


def test_resorted_steps_match_oracle():
    """Steps of a context that re-sorts every step against the oracle, which
    keeps the network in the order as built."""
    n, p0, v0, dt, thr = 2000, 3.8, 0.1, 0.01, 0.1
    xs, ys, th, Lr, Lx, Ly = seeds(n, 10)
    sim = cg.AVM(n, Lr, Lr, xs, ys, th, p0=p0, v0=v0, dt=dt, t1_threshold=thr, seed=11, sort_every=1)
    sim.step(5)
    net, oth, total = oracle.avm_build(xs, ys, Lx, Ly), th, 0
    for s in range(5):
        net, oth, k = oracle.avm_step(net, oth, p0, v0, seed=11, step=s, dt=dt, thr=thr)
        total += k
    hx, hy, gth = (t.cpu().numpy() for t in sim.state())
    vc, vn, cc, cv = (t.cpu().numpy().reshape(-1) for t in sim.topology())
    np.testing.assert_array_equal(vc, net.vc)
    np.testing.assert_array_equal(vn, net.vn)
    np.testing.assert_array_equal(cc, net.cc)
    np.testing.assert_array_equal(cv, net.cv)
    d = (hx - net.hx + Lx / 2) % Lx - Lx / 2
    assert np.abs(d).max() <= 5e-12 * Lx
    np.testing.assert_allclose(gth, oth, rtol=0, atol=5e-13)
    assert total > 0 and sim.counters()["t1_total"] == total
    sim.close()


def test_state_moves_between_sorted_and_unsorted_contexts():
    """A state saved from a re-sorting context loads into another (the load
    puts slots back in tag order) and both continue bit for bit."""
    n = 2000
    xs, ys, th, Lr, Lx, Ly = seeds(n, 13)
    kw = dict(t1_threshold=0.08, seed=3)
    a = cg.AVM(n, Lr, Lr, xs, ys, th, sort_every=3, **kw)
    a.step(20)
    hx, hy, theta = (t.clone() for t in a.state())
    topo = [t.clone() for t in a.topology()]
    step = a.counters()["steps"]
    b = cg.AVM(n, Lr, Lr, xs, ys, th, sort_every=5, **kw)
    b.step(3)
    b.set_state(hx, hy, theta, *topo)
    b.set_step(step)
    c = cg.AVM(n, Lr, Lr, xs, ys, th, **kw)
    c.set_state(hx, hy, theta, *topo)
    c.set_step(step)
    for s in (a, b, c):
        s.step(30)
    for x, y, z in zip(outputs(a), outputs(b), outputs(c)):
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)
    for s in (a, b, c):
        s.close()


def test_full_size_resort_is_bit_identical():
    """N = 65536 (131072 vertices), the benchmark's workload, 300 steps
    re-sorted every 100 against never."""
    n = 65536
    x, y, th, L = workloads.spv_uniform(n, 1)
    kw = dict(p0=3.8, v0=0.1, t1_threshold=0.04, seed=1)
    a = cg.AVM(n, L, L, x, y, th, **kw)
    b = cg.AVM(n, L, L, x, y, th, sort_every=100, **kw)
    a.step(300)
    b.step(300)
    assert_identical(a, b)
    assert a.counters()["t1_total"] > 1000
    a.close()
    b.close()
