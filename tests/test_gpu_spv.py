"""GPU parity of the SPV path against the CPU oracle, through the C ABI.

Sussman, arXiv 1702.02939: topology (Sec. 2.C.3-4) must be bit-exact from the
same state; forces (Eqs. A6-A16) within 1e-10 of max|F|; positions after one
step (Eq. 3) within 1e-12 L.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1702_02939_gb300 as cg  # noqa: E402  (fails loudly if the library is missing)

F_TOL = 1e-10
X_TOL = 1e-12


def make(n, iseed, p0=3.8, v0=0.05, L=None, **kw):
    x, y, th, Lr = workloads.spv_uniform(n, iseed, L)
    Lx, Ly, q = oracle.box(Lr)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    sim = cg.SPV([dict(n=n, Lx=Lr, Ly=Lr, p0=p0, v0=v0)], xs, ys, th, **kw)
    return sim, xs, ys, th, Lx, Ly


def wrapdiff(a, b, L):
    return (a - b + L / 2) % L - L / 2


def check_topology(sim, xs, ys, Lx, Ly):
    cnt, nbr = sim.neighbors()
    topo = oracle.triangulate(xs, ys, Lx, Ly)
    np.testing.assert_array_equal(cnt.cpu().numpy(), topo.cnt)
    np.testing.assert_array_equal(nbr.cpu().numpy(), topo.nbr)
    # the library uses minimum-image neighbours: the oracle's image offsets must agree
    n = len(xs)
    for i in range(0, n, max(1, n // 500)):
        for a in range(topo.cnt[i]):
            j = topo.nbr[i, a]
            dx = xs[j] + topo.off[i, a, 0] * Lx - xs[i]
            dy = ys[j] + topo.off[i, a, 1] * Ly - ys[i]
            assert abs(dx) < Lx / 2 and abs(dy) < Ly / 2
    return topo


@pytest.mark.parametrize("n,seed", [(64, 1), (400, 2), (1000, 3), (4096, 4)])
def test_initial_triangulation_bit_exact(n, seed):
    sim, xs, ys, th, Lx, Ly = make(n, seed)
    check_topology(sim, xs, ys, Lx, Ly)
    sim.close()


@pytest.mark.parametrize("n,seed,p0", [(400, 5, 3.8), (4096, 6, 3.85), (1000, 7, 4.1)])
def test_geometry_and_forces(n, seed, p0):
    sim, xs, ys, th, Lx, Ly = make(n, seed, p0=p0)
    topo = check_topology(sim, xs, ys, Lx, Ly)
    A, P = sim.geometry()
    Fx, Fy, E = sim.forces()
    oFx, oFy, oA, oP, oE = oracle.forces(xs, ys, Lx, Ly, topo, p0)
    np.testing.assert_allclose(A.cpu().numpy(), oA, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(P.cpu().numpy(), oP, rtol=1e-12, atol=1e-13)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    assert np.abs(Fy.cpu().numpy() - oFy).max() <= F_TOL * scale
    assert abs(E - oE) <= 1e-11 * abs(oE)
    sim.close()


@pytest.mark.parametrize("n,seed,v0", [(400, 8, 0.05), (4096, 9, 0.1)])
def test_one_step(n, seed, v0):
    sim, xs, ys, th, Lx, Ly = make(n, seed, p0=3.85, v0=v0, seed=17, dt=0.01)
    sim.step(1)
    gx, gy, gth = (t.cpu().numpy() for t in sim.state())
    ox, oy, oth, _ = oracle.spv_run(xs, ys, th, Lx, Ly, 3.85, v0, 1, seed=17, dt=0.01)
    assert np.abs(wrapdiff(gx, ox, Lx)).max() <= X_TOL * Lx
    assert np.abs(wrapdiff(gy, oy, Ly)).max() <= X_TOL * Ly
    np.testing.assert_allclose(gth, oth, rtol=0, atol=1e-12)
    # topology after the step (test + repair) equals the exact triangulation
    check_topology(sim, gx, gy, Lx, Ly)
    sim.close()


def test_many_steps_keep_exact_delaunay():
    """200 steps of the N=400 workload (p0=3.8, v0=0.05): after every 50 steps
    the maintained rings equal the oracle's triangulation from scratch."""
    sim, xs, ys, th, Lx, Ly = make(400, 1, p0=3.8, v0=0.05, seed=1, dt=0.01)
    for _ in range(4):
        sim.step(50)
        gx, gy, _ = (t.cpu().numpy() for t in sim.state())
        check_topology(sim, gx, gy, Lx, Ly)
    c = sim.counters()
    assert c["steps"] == 200 and c["status"] == 0
    sim.close()


def test_fluid_regime_repairs():
    """Fluid regime with fast cells: many neighbour changes per step."""
    sim, xs, ys, th, Lx, Ly = make(2000, 12, p0=4.0, v0=1.0, seed=3, dt=0.02)
    for _ in range(5):
        sim.step(20)
        gx, gy, _ = (t.cpu().numpy() for t in sim.state())
        check_topology(sim, gx, gy, Lx, Ly)
    c = sim.counters()
    assert c["flagged_total"] > 0
    sim.close()


def test_square_lattice_tie_break_matches_oracle():
    x, y, L = workloads.square_lattice(12)
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    sim = cg.SPV([dict(n=len(xs), Lx=L, Ly=L, p0=3.8, v0=0.0)], xs, ys, np.zeros(len(xs)))
    check_topology(sim, xs, ys, Lx, Ly)
    sim.close()


def test_hexagonal_lattice_zero_force():
    x, y, Lx, Ly = workloads.triangular_lattice(16, 16)
    Lxs, Lys, q = oracle.box(Lx, Ly)
    xs, ys = oracle.snap_positions(x, y, Lxs, Lys)
    sim = cg.SPV([dict(n=len(xs), Lx=Lx, Ly=Ly, p0=3.9, v0=0.0)], xs, ys, np.zeros(len(xs)))
    cnt, nbr = sim.neighbors()
    assert set(cnt.cpu().numpy().tolist()) == {6}
    Fx, Fy, E = sim.forces()
    assert float(Fx.abs().max()) < 1e-12 and float(Fy.abs().max()) < 1e-12
    A, P = sim.geometry()
    np.testing.assert_allclose((P / A.sqrt()).cpu().numpy(), np.sqrt(8 * np.sqrt(3)), rtol=1e-12)
    sim.close()


def test_invalid_positions_raise():
    n = 64
    x, y, th, L = workloads.spv_uniform(n, 1)
    x = x.copy()
    x[3] = 5 * L
    with pytest.raises(cg.CellgbError):
        cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.8, v0=0.05)], x, y, th)


def test_set_p0_v0_change_forces_and_motion():
    sim, xs, ys, th, Lx, Ly = make(400, 21, p0=3.8, v0=0.0)
    topo = oracle.triangulate(xs, ys, Lx, Ly)
    p0 = np.random.default_rng(0).uniform(3.7, 3.9, 400)
    sim.set_p0(p0)
    Fx, Fy, E = sim.forces()
    oFx, oFy, *_ = oracle.forces(xs, ys, Lx, Ly, topo, p0)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    v0 = np.random.default_rng(1).uniform(0.0, 0.3, 400)
    sim.set_v0(v0)
    sim.step(1)
    gx, gy, gth = (t.cpu().numpy() for t in sim.state())
    ox, oy, oth, _ = oracle.spv_run(xs, ys, th, Lx, Ly, p0, v0, 1, seed=0, dt=0.01)
    assert np.abs(wrapdiff(gx, ox, Lx)).max() <= X_TOL * Lx
    sim.close()


def test_full_size_workload():
    """N = 262144, L = 512 (the benchmark workload): initial topology
    bit-exact, forces within tolerance, positions and directors after one
    graph step within tolerance of the oracle's step, and after 10
    fluid-regime steps the maintained topology equals the exact
    triangulation of the new positions."""
    n = 262144
    sim, xs, ys, th, Lx, Ly = make(n, 1, p0=3.85, v0=0.1, seed=1, dt=0.01)
    topo = check_topology(sim, xs, ys, Lx, Ly)
    Fx, Fy, E = sim.forces()
    oFx, oFy, *_ = oracle.forces(xs, ys, Lx, Ly, topo, 3.85)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    assert np.abs(Fy.cpu().numpy() - oFy).max() <= F_TOL * scale
    sim.step(1)
    gx, gy, gth = (t.cpu().numpy() for t in sim.state())
    ox, oy, oth, _ = oracle.spv_run(xs, ys, th, Lx, Ly, 3.85, 0.1, 1, seed=1, dt=0.01)
    assert np.abs(wrapdiff(gx, ox, Lx)).max() <= X_TOL * Lx
    assert np.abs(wrapdiff(gy, oy, Ly)).max() <= X_TOL * Ly
    np.testing.assert_allclose(gth, oth, rtol=0, atol=1e-12)
    sim.step(9)
    gx, gy, _ = (t.cpu().numpy() for t in sim.state())
    check_topology(sim, gx, gy, Lx, Ly)
    sim.close()


def test_hilbert_resort_leaves_results_bit_identical():
    """Re-sorting the storage order (Sec. 2.B) must not change any result:
    rings are canonical by cell index and every sum runs in ring order."""
    n, Lr = 2000, None
    x, y, th, L = workloads.spv_uniform(n, 41)
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    a = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.9, v0=0.3)], xs, ys, th, seed=2, sort_every=0)
    b = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.9, v0=0.3)], xs, ys, th, seed=2, sort_every=7)
    a.step(60)
    b.step(60)
    for ta, tb in zip(a.state(), b.state()):
        assert torch.equal(ta, tb)
    for ta, tb in zip(a.neighbors(), b.neighbors()):
        assert torch.equal(ta, tb)
    fa, fb = a.forces(), b.forces()
    assert torch.equal(fa[0], fb[0]) and torch.equal(fa[1], fb[1])
    gx, gy, _ = (t.cpu().numpy() for t in b.state())
    check_topology(b, gx, gy, Lx, Ly)
    a.close()
    b.close()


def test_batched_replicas_match_per_replica_oracle():
    """Several independent systems of uneven size, box, p0 and v0 in one
    context: each replica equals the oracle run on that replica alone."""
    specs = [(300, 0.0, 3.7, 0.05), (1000, 5.0, 3.95, 0.3), (4096, 0.0, 3.85, 0.1), (700, 2.0, 4.05, 0.5)]
    reps, xs_all, ys_all, th_all, boxes = [], [], [], [], []
    for k, (n, extra, p0, v0) in enumerate(specs):
        x, y, th, L = workloads.spv_uniform(n, 50 + k, None if not extra else (n ** 0.5 + extra))
        Lx, Ly, q = oracle.box(L)
        xs, ys = oracle.snap_positions(x, y, Lx, Ly)
        reps.append(dict(n=n, Lx=L, Ly=L, p0=p0, v0=v0))
        xs_all.append(xs); ys_all.append(ys); th_all.append(th); boxes.append((Lx, Ly))
    sim = cg.SPV(reps, np.concatenate(xs_all), np.concatenate(ys_all), np.concatenate(th_all), seed=9)
    cnt, nbr = (t.cpu().numpy() for t in sim.neighbors())
    Fx, Fy, E = sim.forces()
    Fx, Fy = Fx.cpu().numpy(), Fy.cpu().numpy()
    sim.step(1)
    gx, gy, gth = (t.cpu().numpy() for t in sim.state())
    off = 0
    for k, (n, extra, p0, v0) in enumerate(specs):
        Lx, Ly = boxes[k]
        sl = slice(off, off + n)
        topo = oracle.triangulate(xs_all[k], ys_all[k], Lx, Ly)
        np.testing.assert_array_equal(cnt[sl], topo.cnt)
        local = np.where(nbr[sl] >= 0, nbr[sl] - off, -1)
        np.testing.assert_array_equal(local, topo.nbr)
        oFx, oFy, *_ = oracle.forces(xs_all[k], ys_all[k], Lx, Ly, topo, p0)
        scale = max(np.abs(oFx).max(), np.abs(oFy).max())
        assert np.abs(Fx[sl] - oFx).max() <= F_TOL * scale
        assert np.abs(Fy[sl] - oFy).max() <= F_TOL * scale
        # noise counters use the global cell index of the concatenated
        # system: replica k's cells are tags off ... off + n - 1
        ox, oy, oth = oracle.integrate(xs_all[k], ys_all[k], th_all[k], oFx, oFy, Lx, Ly, v0, 1.0, 1.0, 0.01,
                                       9, 0, tag0=off)
        assert np.abs(wrapdiff(gx[sl], ox, Lx)).max() <= X_TOL * Lx
        assert np.abs(wrapdiff(gy[sl], oy, Ly)).max() <= X_TOL * Ly
        np.testing.assert_allclose(gth[sl], oth, rtol=0, atol=1e-12)
        off += n
    sim.close()


def test_large_force_move_wraps_and_repairs():
    """Two nearly coincident cells feel a very large force; the move of several
    box lengths is wrapped modulo L exactly as in the oracle and the topology
    is repaired to the exact triangulation."""
    n = 256
    x, y, th, L = workloads.spv_uniform(n, 77)
    x = x.copy(); y = y.copy()
    x[1] = x[0] + 1e-5
    y[1] = y[0] + 2e-5
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    sim = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.8, v0=0.1)], xs, ys, th, seed=4, dt=0.01)
    Fx, Fy, E = sim.forces()
    assert float(Fx.abs().max()) * 0.01 > L  # the step moves a cell farther than the box
    sim.step(1)
    gx, gy, gth = (t.cpu().numpy() for t in sim.state())
    ox, oy, oth, _ = oracle.spv_run(xs, ys, th, Lx, Ly, 3.8, 0.1, 1, seed=4, dt=0.01)
    assert np.abs(wrapdiff(gx, ox, Lx)).max() <= 1e-9 * Lx
    assert np.abs(wrapdiff(gy, oy, Ly)).max() <= 1e-9 * Ly
    check_topology(sim, gx, gy, Lx, Ly)
    sim.close()


def ensemble(values):
    v = np.asarray(values, np.float64)
    return v.mean(), v.std(ddof=1) / np.sqrt(len(v))


def test_long_run_ensemble_statistics_match_oracle():
    """Long runs (N = 400, p0 = 3.85, v0 = 0.1, 600 steps of dt = 0.01, eight
    seeds): the ensemble mean shape index q = P / sqrt(A) agrees within 1% and
    the mean-squared displacement within its seed-to-seed standard error.
    Trajectories are compared only through these statistics."""
    n, K, p0, v0 = 400, 600, 3.85, 0.1
    qg, qo, mg, mo = [], [], [], []
    for s in range(8):
        sim, xs, ys, th, Lx, Ly = make(n, 100 + s, p0=p0, v0=v0, seed=s, dt=0.01)
        sim.step(K)
        gx, gy, _ = (t.cpu().numpy() for t in sim.state())
        A, P = (t.cpu().numpy() for t in sim.geometry())
        sim.close()
        ox, oy, _, _ = oracle.spv_run(xs, ys, th, Lx, Ly, p0, v0, K, seed=s, dt=0.01)
        oA, oP, _, _ = oracle.geometry(ox, oy, Lx, Ly, oracle.triangulate(ox, oy, Lx, Ly))
        qg.append((P / np.sqrt(A)).mean())
        qo.append((oP / np.sqrt(oA)).mean())
        mg.append((wrapdiff(gx, xs, Lx) ** 2 + wrapdiff(gy, ys, Ly) ** 2).mean())
        mo.append((wrapdiff(ox, xs, Lx) ** 2 + wrapdiff(oy, ys, Ly) ** 2).mean())
    Qg, _ = ensemble(qg)
    Qo, _ = ensemble(qo)
    Mg, seg = ensemble(mg)
    Mo, seo = ensemble(mo)
    print(f"q: gpu {Qg:.6f} oracle {Qo:.6f}; MSD: gpu {Mg:.6f} +- {seg:.2e} oracle {Mo:.6f} +- {seo:.2e}")
    assert abs(Qg - Qo) <= 0.01 * Qo
    assert abs(Mg - Mo) <= max(seg, seo)


def test_profiled_steps_equal_graph_steps():
    """cg_profile_step (eager launches, repair rounds unrolled to the cap)
    advances the state bit-identically to the graph step, whose repair rounds
    run in a conditional loop node that stops at the first clean round."""
    n = 4096
    a, xs, ys, th, Lx, Ly = make(n, 31, p0=3.85, v0=0.1, seed=2)
    b, *_ = make(n, 31, p0=3.85, v0=0.1, seed=2)
    a.step(25)
    b.profile(25)
    for ta, tb in zip(a.state(), b.state()):
        assert torch.equal(ta, tb)
    for ta, tb in zip(a.neighbors(), b.neighbors()):
        assert torch.equal(ta, tb)
    ca, cb = a.counters(), b.counters()
    for k in ("steps", "flagged_total", "repaired_total", "status"):
        assert ca[k] == cb[k]
    # the loop ran at least one round per step, and at most the cap
    assert 25 <= ca["loop_total"] <= 25 * 4
    a.close()
    b.close()


def test_repair_cap_status():
    """From a random state the first step needs more than one repair round:
    with repair_cap = 1 the loop stops and the host sees CG_EREPAIR_CAP."""
    sim, *_ = make(4096, 32, p0=3.85, v0=0.1, repair_cap=1)
    with pytest.raises(cg.CellgbError) as e:
        sim.step(1)
        sim.sync()
    assert e.value.code == -4
    sim.close()


def test_launch_shapes_do_not_change_results():
    """Grids of the repair, check and director kernels, the node priorities
    and the ring-size grouping of the geometry and force passes change timing
    only: 20 steps agree bit for bit."""
    n = 4096
    a, *_ = make(n, 33, p0=3.85, v0=0.1, seed=3)
    assert a.launch["ring_order"] == 5 and a.launch["force_beside"] == 0
    b, *_ = make(n, 33, p0=3.85, v0=0.1, seed=3)
    b.set_launch(repair_blocks_per_sm=8, check_blocks_per_sm=4, dir_blocks_per_sm=1, dir_low_priority=1,
                 geom_blocks_per_sm=2, test_blocks_per_sm=2, ring_order=0, dir_beside_geom=0, force_beside=0)
    assert b.launch["dir_blocks_per_sm"] == 1
    c, *_ = make(n, 33, p0=3.85, v0=0.1, seed=3)
    c.set_launch(dir_beside_geom=1, dir_low_priority=0, dir_blocks_per_sm=0, ring_order=3)
    assert c.launch["dir_beside_geom"] == 1
    d, *_ = make(n, 33, p0=3.85, v0=0.1, seed=3)
    d.set_launch(ring_order=6, force_beside=1)
    a.step(20)
    b.step(20)
    c.step(20)
    d.step(20)
    for ta, tb, tc, td in zip(a.state() + a.neighbors() + a.forces()[:2], b.state() + b.neighbors() + b.forces()[:2],
                              c.state() + c.neighbors() + c.forces()[:2], d.state() + d.neighbors() + d.forces()[:2]):
        assert torch.equal(ta, tb) and torch.equal(ta, tc) and torch.equal(ta, td)
    with pytest.raises(RuntimeError):
        c.set_launch(dir_beside_geom=2)
    with pytest.raises(RuntimeError):
        c.set_launch(ring_order=8)
    with pytest.raises(RuntimeError):
        c.set_launch(force_beside=2)
    for s in (a, b, c, d):
        s.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_force_pass_beside_the_rounds_keeps_results(precision):
    """The force pass run beside the repair rounds, with the cells around
    rewritten rings (and any it could not decide) done again afterwards,
    gives bit for bit the state of the force pass after the rounds, in a
    regime that rewrites many rings every step, in FP64 and FP32 mode."""
    n = 16384
    a, *_ = make(n, 35, p0=3.95, v0=0.5, seed=5, precision=precision)
    b, *_ = make(n, 35, p0=3.95, v0=0.5, seed=5, precision=precision)
    a.set_launch(force_beside=1)
    b.set_launch(force_beside=0)
    a.step(60)
    b.step(60)
    ca, cb = a.counters(), b.counters()
    assert ca["repaired_total"] > 60 * 20 and ca == cb
    for ta, tb in zip(a.state() + a.neighbors() + a.forces()[:2], b.state() + b.neighbors() + b.forces()[:2]):
        assert torch.equal(ta, tb)
    a.close()
    b.close()


def test_autotune_takes_no_step_and_keeps_results():
    """The autotuner times candidates on a temporary copy: the context's state
    and step counter are untouched and later steps equal an untuned run."""
    n = 4096
    a, *_ = make(n, 34, p0=3.85, v0=0.1, seed=4)
    b, *_ = make(n, 34, p0=3.85, v0=0.1, seed=4)
    a.step(3)
    b.step(3)
    before = a.state()
    best, ms = a.autotune(3)
    assert ms > 0 and set(best) == {"repair_blocks_per_sm", "check_blocks_per_sm", "dir_blocks_per_sm",
                                    "dir_low_priority", "geom_blocks_per_sm", "test_blocks_per_sm",
                                    "dir_beside_geom", "ring_order", "force_beside"}
    assert a.launch == best
    for t0, t1 in zip(before, a.state()):
        assert torch.equal(t0, t1)
    assert a.counters()["steps"] == 3
    a.step(10)
    b.step(10)
    for ta, tb in zip(a.state() + a.neighbors(), b.state() + b.neighbors()):
        assert torch.equal(ta, tb)
    a.close()
    b.close()


def test_autotune_cache_reuses_a_tuning(tmp_path):
    """A tuning stored in a cache file is applied by the next context of the
    same problem class without timing; results stay those of any shapes."""
    path = str(tmp_path / "launch.json")
    n = 4096
    a, *_ = make(n, 36, p0=3.85, v0=0.1, seed=5)
    best, ms = a.autotune(2, cache=path)
    assert ms is not None
    b, *_ = make(n, 36, p0=3.85, v0=0.1, seed=5)
    again, ms2 = b.autotune(2, cache=path)
    assert ms2 is None and again == best and b.launch == best
    c, *_ = make(n, 36, p0=3.85, v0=0.1, seed=5)
    a.step(5)
    b.step(5)
    c.step(5)
    for ta, tb, tc in zip(a.state(), b.state(), c.state()):
        assert torch.equal(ta, tb) and torch.equal(ta, tc)
    for s in (a, b, c):
        s.close()


# FP32 mode (single-precision physics, exact topology).  Bounds from the
# arithmetic: every FP32 operation rounds with relative error u = 2^-24; the
# force on a cell is a chain of about 30 dependent operations (relative
# positions, circumcentres, edge vectors and lengths, force sets, Jacobian
# factors and their sum over the ring) whose terms are up to ~10x larger than
# the result, so |F32 - F64| <= 30 u * 10 * max|F| ~ 2e-5 max|F|; the noise
# uses 24-bit uniforms and FP32 log/cos (relative 1e-6), so theta after one
# step is within sqrt(2 D_r dt) * 6 * 1e-6 < 1e-5.
F32_TOL = 2e-5


@pytest.mark.parametrize("n,seed", [(400, 41), (4096, 42)])
def test_fp32_mode_topology_forces_and_step(n, seed):
    sim, xs, ys, th, Lx, Ly = make(n, seed, p0=3.85, v0=0.1, seed=3, dt=0.01, precision="f32")
    topo = check_topology(sim, xs, ys, Lx, Ly)  # exact predicates: bit-exact
    Fx, Fy, _ = sim.forces()
    oFx, oFy, oA, oP, _ = oracle.forces(xs, ys, Lx, Ly, topo, 3.85)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    errF = max(np.abs(Fx.cpu().numpy() - oFx).max(), np.abs(Fy.cpu().numpy() - oFy).max()) / scale
    A, P = (t.cpu().numpy() for t in sim.geometry())
    errA = np.abs(A - oA).max() / np.abs(oA).max()
    errP = np.abs(P - oP).max() / np.abs(oP).max()
    print(f"fp32 n={n}: force err {errF:.2e} max|F|, A {errA:.2e}, P {errP:.2e}")
    assert errF <= F32_TOL
    assert errA <= 1e-5 and errP <= 1e-5
    sim.step(1)
    gx, gy, gth = (t.cpu().numpy() for t in sim.state())
    ox, oy, oth, _ = oracle.spv_run(xs, ys, th, Lx, Ly, 3.85, 0.1, 1, seed=3, dt=0.01)
    xtol = 0.01 * F32_TOL * scale + X_TOL * Lx
    assert np.abs(wrapdiff(gx, ox, Lx)).max() <= xtol
    assert np.abs(wrapdiff(gy, oy, Ly)).max() <= xtol
    assert np.abs(gth - oth).max() <= 1e-5
    sim.close()


def test_fp32_mode_long_run_statistics():
    """FP32 trajectories leave the FP64 ones after a few hundred steps (the
    dynamics amplify the rounding differences); the ensemble statistics still
    agree: mean shape index within 1% and MSD within three combined standard
    errors (eight seeds, N = 400, p0 = 3.85, v0 = 0.1, 600 steps)."""
    n, K, p0, v0 = 400, 600, 3.85, 0.1
    qg, qo, mg, mo = [], [], [], []
    for s in range(8):
        sim, xs, ys, th, Lx, Ly = make(n, 300 + s, p0=p0, v0=v0, seed=s, dt=0.01, precision="f32")
        sim.step(K)
        gx, gy, _ = (t.cpu().numpy() for t in sim.state())
        A, P = (t.cpu().numpy() for t in sim.geometry())
        sim.close()
        ox, oy, _, _ = oracle.spv_run(xs, ys, th, Lx, Ly, p0, v0, K, seed=s, dt=0.01)
        oA, oP, _, _ = oracle.geometry(ox, oy, Lx, Ly, oracle.triangulate(ox, oy, Lx, Ly))
        qg.append((P / np.sqrt(A)).mean())
        qo.append((oP / np.sqrt(oA)).mean())
        mg.append((wrapdiff(gx, xs, Lx) ** 2 + wrapdiff(gy, ys, Ly) ** 2).mean())
        mo.append((wrapdiff(ox, xs, Lx) ** 2 + wrapdiff(oy, ys, Ly) ** 2).mean())
    Qg, _ = ensemble(qg)
    Qo, _ = ensemble(qo)
    Mg, seg = ensemble(mg)
    Mo, seo = ensemble(mo)
    print(f"fp32 q: {Qg:.6f} vs {Qo:.6f}; MSD {Mg:.6f} +- {seg:.2e} vs {Mo:.6f} +- {seo:.2e}")
    assert abs(Qg - Qo) <= 0.01 * Qo
    assert abs(Mg - Mo) <= 3.0 * np.hypot(seg, seo)


def test_fp32_mode_refuses_the_backward_pass():
    sim, *_ = make(400, 43, precision="f32")
    with pytest.raises(cg.CellgbError) as e:
        sim.hvp(np.zeros(400), np.zeros(400))
    assert e.value.code == -1
    sim.close()


def test_host_side_fault_injection_gives_clean_errors():
    """Faults injected on the host come back as status codes, never as a
    GPU fault: non-finite parameters or directors at creation, a non-finite
    p0 later, a box too small for the Voronoi search."""
    n = 64
    x, y, th, L = workloads.spv_uniform(n, 2)
    rep = [dict(n=n, Lx=L, Ly=L, p0=3.8, v0=0.05)]
    with pytest.raises(cg.CellgbError) as e:
        cg.SPV(rep, x, y, th, KA=float("nan"))
    assert e.value.code == -1
    bad = th.copy()
    bad[5] = float("inf")
    with pytest.raises(cg.CellgbError) as e:
        cg.SPV(rep, x, y, bad)
    assert e.value.code == -1
    sim = cg.SPV(rep, x, y, th)
    p0 = np.full(n, 3.8)
    p0[7] = float("nan")
    with pytest.raises(cg.CellgbError) as e:
        sim.set_p0(p0)
    assert e.value.code == -1
    sim.close()
    x16, y16, th16, L16 = workloads.spv_uniform(16, 1)
    with pytest.raises(cg.CellgbError) as e:
        cg.SPV([dict(n=16, Lx=L16, Ly=L16, p0=3.8, v0=0.05)], x16, y16, th16)
    assert e.value.code == -7


def test_checkpoint_and_resume_is_bit_identical():
    """A run saved after 15 steps (positions, directors, p0, v0, step counter)
    and resumed in a fresh context continues exactly like the uninterrupted
    run: Philox noise is counter based and the topology is rebuilt exactly."""
    n = 4096
    a, xs, ys, th, Lx, Ly = make(n, 35, p0=3.85, v0=0.1, seed=9)
    p0 = np.random.default_rng(4).uniform(3.7, 4.0, n)
    a.set_p0(p0)
    a.step(15)
    x15, y15, th15 = a.state()
    b = cg.SPV([dict(n=n, Lx=Lx, Ly=Ly, p0=3.85, v0=0.1)], x15, y15, th15, seed=9)
    b.set_p0(p0)
    b.set_step(15)
    a.step(25)
    b.step(25)
    for ta, tb in zip(a.state() + a.neighbors(), b.state() + b.neighbors()):
        assert torch.equal(ta, tb)
    assert a.counters()["steps"] == b.counters()["steps"] == 40
    a.close()
    b.close()


def test_rectangular_box():
    """Lx != Ly (aspect 2.5): the minimum image and the cell list work per
    axis; topology bit-exact, forces and one step within tolerance, and after
    20 steps the maintained topology is the exact triangulation."""
    n, Lxr, Lyr = 1000, 50.0, 20.0
    x, y, th = workloads.spv_uniform_rect(n, 44, Lxr, Lyr)
    Lx, Ly, q = oracle.box(Lxr, Lyr)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    sim = cg.SPV([dict(n=n, Lx=Lxr, Ly=Lyr, p0=3.85, v0=0.1)], xs, ys, th, seed=6)
    topo = check_topology(sim, xs, ys, Lx, Ly)
    Fx, Fy, _ = sim.forces()
    oFx, oFy, *_ = oracle.forces(xs, ys, Lx, Ly, topo, 3.85)
    scale = max(np.abs(oFx).max(), np.abs(oFy).max())
    assert np.abs(Fx.cpu().numpy() - oFx).max() <= F_TOL * scale
    assert np.abs(Fy.cpu().numpy() - oFy).max() <= F_TOL * scale
    sim.step(1)
    gx, gy, _ = (t.cpu().numpy() for t in sim.state())
    ox, oy, _, _ = oracle.spv_run(xs, ys, th, Lx, Ly, 3.85, 0.1, 1, seed=6)
    assert np.abs(wrapdiff(gx, ox, Lx)).max() <= X_TOL * Lx
    assert np.abs(wrapdiff(gy, oy, Ly)).max() <= X_TOL * Ly
    sim.step(20)
    gx, gy, _ = (t.cpu().numpy() for t in sim.state())
    check_topology(sim, gx, gy, Lx, Ly)
    sim.close()


def test_director_terms_match_libm_and_oracle():
    """n(theta) and the Box-Muller noise of Eq. 3 as the FP64 step evaluates
    them (table-driven sin, cos and ln) against numpy's sin/cos and the
    oracle's noise.  Angles include the table points j pi/128 and their
    neighbourhoods, multiples of pi/2, tiny and large |theta|, and |theta| >=
    2^20 (evaluated by CUDA's sincos)."""
    sim, *_ = make(64, 41, seed=123)
    rng = np.random.default_rng(17)
    parts = [
        rng.uniform(-50.0, 50.0, 40000),
        rng.uniform(-2e5, 2e5, 20000),
        np.arange(-3000, 3000) * (np.pi / 128),
        np.arange(-3000, 3000) * (np.pi / 128) + rng.uniform(-1e-9, 1e-9, 6000),
        np.arange(-200, 200) * (np.pi / 2),
        rng.uniform(-1e-6, 1e-6, 2000),
        np.array([0.0, -0.0, 2.0 ** -1074, 2.0 ** 20 - 1e-6, 2.0 ** 20, -(2.0 ** 20), 3e7, -1e9]),
    ]
    th = np.concatenate(parts)
    n = len(th)
    tag = rng.integers(0, 2 ** 31 - 1, n, dtype=np.int64).astype(np.int32)
    step = 987654321
    cs, sn, xi = sim.director_terms(torch.from_numpy(th), torch.from_numpy(tag), step)
    cs, sn, xi = cs.cpu().numpy(), sn.cpu().numpy(), xi.cpu().numpy()
    ulp = 2.0 ** -53
    # libm is within 1 ulp, the table method within 4 units of 2^-53 (absolute)
    assert np.max(np.abs(cs - np.cos(th))) <= 6 * ulp
    assert np.max(np.abs(sn - np.sin(th))) <= 6 * ulp
    assert np.max(np.abs(cs * cs + sn * sn - 1.0)) <= 8 * ulp
    # exact where the angle is exactly 0
    assert cs[-8] == 1.0 and sn[-8] == 0.0 and sn[-7] == 0.0
    # xi = R cos(2 pi u2), R = sqrt(-2 ln u1).  The oracle rounds 2 pi u2 before
    # its cosine (absolute error up to ~7 units of 2^-53 in the cosine), the
    # table method is within 4; both round ln and the product, and the step
    # takes sqrt(x) as x * rsqrt(x) (third-order refined: within 2 ulp of R).
    for k in range(0, n, 7):
        ref = oracle.director_noise(123, int(tag[k]), step)
        r = oracle.philox([int(tag[k]), step & 0xFFFFFFFF, step >> 32, 0], [123, 0])
        u1 = ((((r[0] << 32) | r[1]) >> 11) + 1) * 2.0 ** -53
        R = np.sqrt(-2.0 * np.log(u1))
        assert abs(xi[k] - ref) <= ulp * (16 * R + 8 * abs(ref)), (k, xi[k], ref, R)
    # the noise is a standard normal
    assert abs(xi.mean()) < 0.02 and abs(xi.std() - 1.0) < 0.02
    sim.close()


@pytest.mark.parametrize("precision,sort_every", [("f64", 0), ("f32", 0), ("f64", 3)])
def test_run_io_is_bit_identical_to_set_step_get(precision, sort_every):
    """cg_run_io (uploads overlapped with the steps, double-buffered staging)
    gives the same positions, bit for bit, as cg_set_v0, cg_step(1),
    cg_get_state per step; with a per-step v0 and per-step outputs, and with
    v0 kept and one output buffer reused."""
    n, K = 1000, 7
    kw = dict(p0=3.85, v0=0.1, seed=8, dt=0.01, precision=precision, sort_every=sort_every)
    a, *_ = make(n, 51, **kw)
    b, *_ = make(n, 51, **kw)
    rng = np.random.default_rng(5)
    v0 = rng.uniform(0.0, 0.3, (K, n))
    ref_x, ref_y = [], []
    for k in range(K):
        a.set_v0(v0[k])
        a.step(1)
        x, y, _ = a.state()
        ref_x.append(x.cpu().numpy())
        ref_y.append(y.cpu().numpy())
    hv0 = torch.from_numpy(v0.ravel().copy()).pin_memory()
    hx = torch.empty(K * n, dtype=torch.float64).pin_memory()
    hy = torch.empty(K * n, dtype=torch.float64).pin_memory()
    b.run_io(K, v0=hv0, x=hx, y=hy, v0_stride=n, out_stride=n)
    for k in range(K):
        np.testing.assert_array_equal(hx[k * n:(k + 1) * n].numpy(), ref_x[k])
        np.testing.assert_array_equal(hy[k * n:(k + 1) * n].numpy(), ref_y[k])
    # v0 kept, one reused output buffer (device tensors this time)
    a.step(3)
    dx = torch.empty(n, dtype=torch.float64, device="cuda")
    dy = torch.empty(n, dtype=torch.float64, device="cuda")
    b.run_io(3, x=dx, y=dy)
    x, y, th = a.state()
    assert torch.equal(dx, x) and torch.equal(dy, y)
    # a per-step v0 read in place from device memory, one step and several
    for k in (1, 3):
        for j in range(k):
            a.set_v0(v0[j])
            a.step(1)
        dv0 = torch.from_numpy(v0[:k].ravel().copy()).cuda()
        b.run_io(k, v0=dv0, x=dx, y=dy, v0_stride=n)
        x, y, th = a.state()
        assert torch.equal(dx, x) and torch.equal(dy, y)
    # pageable host buffers (staged copies), one step and several
    for k in (1, 2):
        a.set_v0(v0[k])
        a.step(k)
        px, py = np.empty(k * n), np.empty(k * n)
        b.run_io(k, v0=np.tile(v0[k], k), x=px, y=py, v0_stride=n, out_stride=n)
        x, y, _ = a.state()
        np.testing.assert_array_equal(px[(k - 1) * n:], x.cpu().numpy())
        np.testing.assert_array_equal(py[(k - 1) * n:], y.cpu().numpy())
    for t0, t1 in zip(a.state(), b.state()):
        assert torch.equal(t0, t1)
    a.close()
    b.close()


def test_run_io_refuses_a_non_finite_v0():
    sim, *_ = make(400, 52, seed=2)
    bad = np.full(400, 0.05)
    bad[17] = np.nan
    with pytest.raises(cg.CellgbError) as e:
        sim.run_io(2, v0=bad)
    assert e.value.code == -1  # CG_EINVAL
    # the status read back stays: the next call is refused before any work
    steps = sim.counters()["steps"]
    with pytest.raises(cg.CellgbError) as e:
        sim.run_io(1)
    assert e.value.code == -1 and sim.counters()["steps"] == steps
    sim.close()


def test_run_io_returns_a_status_raised_before_it():
    """cg_run_io does not synchronise on entry: a status raised by earlier,
    still unread work (a step that runs out of repair rounds) is returned
    when the call ends, and the context refuses further I/O steps."""
    sim, *_ = make(4096, 32, p0=3.85, v0=0.1, repair_cap=1)
    sim.step(1)  # enqueued only; its status is not read here
    with pytest.raises(cg.CellgbError) as e:
        sim.run_io(1)
    assert e.value.code == -4
    with pytest.raises(cg.CellgbError) as e:
        sim.run_io(1)
    assert e.value.code == -4
    sim.close()


def test_coincident_cells_are_refused():
    """Two cells at exactly the same position have no Voronoi polygon between
    them: the triangulation refuses the state with CG_EDEGENERATE."""
    n = 400
    x, y, th, L = workloads.spv_uniform(n, 61)
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    xs, ys = xs.copy(), ys.copy()
    xs[7], ys[7] = xs[123], ys[123]
    with pytest.raises(cg.CellgbError) as e:
        cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.8, v0=0.05)], xs, ys, th)
    assert e.value.code == -8


def test_million_cells_sampled_against_local_triangulations():
    """N = 1048576 (the largest size of the timing sweep), 20 fluid steps:
    ring symmetry and 6N ring entries over all cells, areas tiling the box,
    and the rings of the cells inside three windows equal to the exact
    Delaunay triangulation of the window's points computed by the oracle."""
    n = 1 << 20
    sim, xs, ys, th, Lx, Ly = make(n, 71, p0=3.85, v0=0.1, seed=5, dt=0.01)
    sim.step(20)
    cnt, nbr = (t.cpu().numpy() for t in sim.neighbors())
    assert int(cnt.sum()) == 6 * n
    rows = np.repeat(np.arange(n, dtype=np.int64), cnt)
    cols = nbr[nbr >= 0].astype(np.int64)
    # j in ring(i) <=> i in ring(j): the directed edges equal their reverses
    np.testing.assert_array_equal(np.sort(rows * n + cols), np.sort(cols * n + rows))
    A, P = (t.cpu().numpy() for t in sim.geometry())
    assert abs(A.sum() - Lx * Ly) <= 1e-9 * Lx * Ly
    gx, gy, _ = (t.cpu().numpy() for t in sim.state())
    q = oracle.grid_exponent(Lx, Ly)
    X = np.rint(np.ldexp(gx, q)).astype(np.int64)
    Y = np.rint(np.ldexp(gy, q)).astype(np.int64)
    rng = np.random.default_rng(8)
    for _ in range(3):
        cx, cy = rng.uniform(0.25 * Lx, 0.75 * Lx), rng.uniform(0.25 * Ly, 0.75 * Ly)
        hw, margin = 20.0, 8.0
        inside = np.nonzero((np.abs(gx - cx) < hw + margin) & (np.abs(gy - cy) < hw + margin))[0]
        core = set(np.nonzero((np.abs(gx - cx) < hw) & (np.abs(gy - cy) < hw))[0].tolist())
        wcnt, wnbr = oracle.delaunay_plain(X[inside], Y[inside])
        checked = 0
        for k, i in enumerate(inside):
            if int(i) not in core:
                continue
            ring = {int(inside[j]) for j in wnbr[k, :wcnt[k]]}
            assert ring == set(nbr[i, :cnt[i]].tolist()), i
            checked += 1
        assert checked > 1000
    sim.close()


def test_full_size_thousand_steps_stay_exact():
    """The benchmark workload's length: N = 262144, 100 + 1000 graph steps in
    the fluid regime; the maintained topology then equals the oracle's exact
    triangulation of the final positions, and the areas tile the box."""
    n = 262144
    sim, xs, ys, th, Lx, Ly = make(n, 1, p0=3.85, v0=0.1, seed=1, dt=0.01)
    sim.step(1100)
    gx, gy, _ = (t.cpu().numpy() for t in sim.state())
    check_topology(sim, gx, gy, Lx, Ly)
    A, P = (t.cpu().numpy() for t in sim.geometry())
    assert abs(A.sum() - Lx * Ly) <= 1e-9 * Lx * Ly
    assert sim.counters()["status"] == 0
    sim.close()


def test_full_size_batched_replicas_stay_exact():
    """The batched workload at full size: 512 replicas (N_r log-uniform on
    [256, 16384], per-replica p0, v0 and box) in one context, 2000 steps; then
    the rings of six sampled replicas equal the oracle's exact triangulation
    of each replica's final positions, and every replica's areas tile its box."""
    R = 512
    sizes = workloads.replica_sizes(R, 7)
    p0s, v0s = workloads.replica_params(R, 7)
    reps, xs, ys, ths, boxes = [], [], [], [], []
    for r in range(R):
        x, y, th, L = workloads.spv_uniform(int(sizes[r]), 1000 + r)
        reps.append(dict(n=int(sizes[r]), Lx=L, Ly=L, p0=float(p0s[r]), v0=float(v0s[r])))
        xs.append(x); ys.append(y); ths.append(th); boxes.append(oracle.box(L)[:2])
    sim = cg.SPV(reps, np.concatenate(xs), np.concatenate(ys), np.concatenate(ths), dt=0.01, seed=7)
    sim.step(2000)
    gx, gy, _ = (t.cpu().numpy() for t in sim.state())
    cnt, nbr = (t.cpu().numpy() for t in sim.neighbors())
    A, _ = (t.cpu().numpy() for t in sim.geometry())
    assert sim.counters()["status"] == 0
    starts = np.concatenate([[0], np.cumsum(sizes)])
    for r in range(R):
        a, b = starts[r], starts[r + 1]
        Lx, Ly = boxes[r]
        assert abs(A[a:b].sum() - Lx * Ly) <= 1e-9 * Lx * Ly
    for r in np.random.default_rng(3).choice(R, 6, replace=False):
        a, b = starts[r], starts[r + 1]
        Lx, Ly = boxes[r]
        topo = oracle.triangulate(gx[a:b], gy[a:b], Lx, Ly)
        np.testing.assert_array_equal(cnt[a:b], topo.cnt)
        np.testing.assert_array_equal(nbr[a:b] - np.where(nbr[a:b] >= 0, a, 0), topo.nbr)
    sim.close()
