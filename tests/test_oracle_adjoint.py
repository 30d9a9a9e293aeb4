"""Pins the oracle's adjoint of an SPV run.

The step map of Eq. 3 (Sussman, arXiv 1702.02939) with fixed noise has the
transposed Jacobian I - dt mu H, H the Hessian of E (Eq. 1); the oracle gets
H v as the dual-number derivative of its force (Eqs. A6-A16).  Pins: H is
symmetric, H v equals central finite differences of the force, the gradient of
a function of the areas and perimeters equals finite differences, and the full
reverse pass equals central finite differences (h = 1e-6) of the run's loss on
windows where the topology does not change.
"""
import numpy as np
import pytest

import oracle
import workloads


def state(n, seed):
    x, y, th, L = workloads.spv_uniform(n, seed)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    return x, y, th, Lx, Ly


def test_hessian_is_symmetric_and_matches_fd():
    x, y, th, Lx, Ly = state(100, 3)
    topo = oracle.triangulate(x, y, Lx, Ly)
    rng = np.random.default_rng(0)
    u, v = rng.normal(size=(2, 100)), rng.normal(size=(2, 100))
    Hu = oracle.hvp(x, y, Lx, Ly, topo, 3.8, u[0], u[1])
    Hv = oracle.hvp(x, y, Lx, Ly, topo, 3.8, v[0], v[1])
    a = (u[0] * Hv[0] + u[1] * Hv[1]).sum()
    b = (v[0] * Hu[0] + v[1] * Hu[1]).sum()
    assert abs(a - b) <= 1e-10 * abs(a)
    h = 1e-6
    Fp = oracle.forces(x + h * v[0], y + h * v[1], Lx, Ly, topo, 3.8)
    Fm = oracle.forces(x - h * v[0], y - h * v[1], Lx, Ly, topo, 3.8)
    scale = max(np.abs(Hv[0]).max(), np.abs(Hv[1]).max())
    assert np.abs(-(Fp[0] - Fm[0]) / (2 * h) - Hv[0]).max() <= 1e-6 * scale
    assert np.abs(-(Fp[1] - Fm[1]) / (2 * h) - Hv[1]).max() <= 1e-6 * scale
    assert np.abs((Fp[2] - Fm[2]) / (2 * h) - Hv[2]).max() <= 1e-6 * np.abs(Hv[2]).max()
    assert np.abs((Fp[3] - Fm[3]) / (2 * h) - Hv[3]).max() <= 1e-6 * np.abs(Hv[3]).max()


def test_geometry_gradient_matches_fd():
    x, y, th, Lx, Ly = state(64, 4)
    topo = oracle.triangulate(x, y, Lx, Ly)
    rng = np.random.default_rng(1)
    cA, cP = rng.normal(size=64), rng.normal(size=64)
    gx, gy = oracle.geom_grad(x, y, Lx, Ly, topo, cA, cP)

    def f(xx, yy):
        A, P, _, _ = oracle.geometry(xx, yy, Lx, Ly, topo)
        return (cA * A + cP * P).sum()

    h = 1e-6
    for i in range(0, 64, 7):
        e = np.zeros(64)
        e[i] = h
        assert abs((f(x + e, y) - f(x - e, y)) / (2 * h) - gx[i]) <= 1e-6 * np.abs(gx).max()
        assert abs((f(x, y + e) - f(x, y - e)) / (2 * h) - gy[i]) <= 1e-6 * np.abs(gy).max()


def shape_loss(A, P, target=3.95):
    """Mean over cells of (A (P / sqrt(A) - target))^2 and its partials."""
    r = P * np.sqrt(A) - target * A
    n = len(A)
    L = (r * r).mean()
    gA = 2.0 * r * (P / (2.0 * np.sqrt(A)) - target) / n
    gP = 2.0 * r * np.sqrt(A) / n
    return L, gA, gP


def run_loss(x, y, th, Lx, Ly, p0, v0, K, seed, KA=1.0, KP=1.0):
    x1, y1, _, _ = oracle.spv_run(x, y, th, Lx, Ly, p0, v0, K, seed=seed, KA=KA, KP=KP)
    topo = oracle.triangulate(x1, y1, Lx, Ly)
    A, P, _, _ = oracle.geometry(x1, y1, Lx, Ly, topo)
    return shape_loss(A, P)[0], topo


@pytest.mark.parametrize("K", [1, 4])
def test_backward_matches_finite_differences(K):
    n, seed = 64, 11
    x, y, th, Lx, Ly = state(n, 6)
    p0 = np.random.default_rng(2).uniform(3.7, 3.9, n)
    v0 = 0.1
    fwd = oracle.spv_backward(x, y, th, Lx, Ly, p0, v0, K, seed, np.zeros(n), np.zeros(n), np.zeros(n),
                              np.zeros(n))
    L0, gA, gP = shape_loss(fwd["A"], fwd["P"])
    out = oracle.spv_backward(x, y, th, Lx, Ly, p0, v0, K, seed, np.zeros(n), np.zeros(n), gA, gP)
    _, topo0 = run_loss(x, y, th, Lx, Ly, p0, v0, K, seed)
    h = 1e-6

    def fd(fn):
        Lp, tp = fn(+h)
        Lm, tm = fn(-h)
        # only meaningful on topology-stable windows
        assert np.array_equal(tp.nbr, topo0.nbr) and np.array_equal(tm.nbr, topo0.nbr)
        return (Lp - Lm) / (2 * h)

    def close(a, b, scale):
        # 1e-6 relative to the max-norm of that parameter's gradient (as forces
        # are compared relative to max|F|), plus the round-off floor of a
        # central difference with h = 1e-6: ~ eps |L| / h amplified ~100x by
        # the run, i.e. 1e-8 |L|
        assert abs(a - b) <= 1e-6 * scale + 1e-8 * abs(L0), (a, b, scale)

    gpos = max(np.abs(out["gx0"]).max(), np.abs(out["gy0"]).max())
    for i in (0, 17, 40):
        e = np.zeros(n)
        e[i] = 1.0
        close(fd(lambda s: run_loss(x + s * e, y, th, Lx, Ly, p0, v0, K, seed)), out["gx0"][i], gpos)
        close(fd(lambda s: run_loss(x, y + s * e, th, Lx, Ly, p0, v0, K, seed)), out["gy0"][i], gpos)
        close(fd(lambda s: run_loss(x, y, th, Lx, Ly, p0 + s * e, v0, K, seed)), out["gp0"][i],
              np.abs(out["gp0"]).max())
    gv0 = out["gv0"].sum()
    close(fd(lambda s: run_loss(x, y, th, Lx, Ly, p0, v0 + s, K, seed)), gv0, abs(gv0))
    close(fd(lambda s: run_loss(x, y, th, Lx, Ly, p0, v0, K, seed, KA=1.0 + s)), out["gKA"], abs(out["gKA"]))
    close(fd(lambda s: run_loss(x, y, th, Lx, Ly, p0, v0, K, seed, KP=1.0 + s)), out["gKP"], abs(out["gKP"]))
