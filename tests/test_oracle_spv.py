"""Pins the oracle's SPV geometry, forces and integrator against closed forms.

Sussman, arXiv 1702.02939: energy Eq. 1, force Eq. 2 / A6 (F = -grad E),
equation of motion Eq. 3, Voronoi geometry Sec. 2.C.1, appendix A1-A16.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def state(n, seed):
    x, y, th, L = workloads.spv_uniform(n, seed)
    Lx, Ly, q = oracle.box(L)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    return x, y, th, Lx, Ly


@pytest.mark.parametrize("n", [64, 400, 4096])
def test_areas_tile_the_box(n):
    x, y, th, Lx, Ly = state(n, 2)
    topo = oracle.triangulate(x, y, Lx, Ly)
    A, P, hx, hy = oracle.geometry(x, y, Lx, Ly, topo)
    assert np.all(A > 0) and np.all(P > 0)
    assert abs(A.sum() - Lx * Ly) <= 1e-12 * Lx * Ly


@pytest.mark.parametrize("a", [1.0, 0.75])
def test_hexagonal_lattice_closed_forms(a):
    x, y, Lx, Ly = workloads.triangular_lattice(8, 8, a=a)
    Lx, Ly, q = oracle.box(Lx, Ly)
    x, y = oracle.snap_positions(x, y, Lx, Ly)
    topo = oracle.triangulate(x, y, Lx, Ly)
    A, P, _, _ = oracle.geometry(x, y, Lx, Ly, topo)
    # regular hexagon with inradius a/2: area (sqrt3/2) a^2, perimeter 2 sqrt3 a
    np.testing.assert_allclose(A, math.sqrt(3) / 2 * a * a, rtol=1e-12)
    np.testing.assert_allclose(P, 2 * math.sqrt(3) * a, rtol=1e-12)
    np.testing.assert_allclose(P / np.sqrt(A), math.sqrt(8 * math.sqrt(3)), rtol=1e-12)
    for p0 in (3.5, 3.8, 4.2):
        Fx, Fy, *_ = oracle.forces(x, y, Lx, Ly, topo, p0)
        # symmetry: every cell sees the same environment -> zero net force
        assert np.abs(Fx).max() < 1e-12 and np.abs(Fy).max() < 1e-12


def fd_check(x, y, Lx, Ly, topo, p0, A0, KA, KP, cells, h=1e-6):
    Fx, Fy, *_ = oracle.forces(x, y, Lx, Ly, topo, p0, A0, KA, KP)
    scale = max(np.abs(Fx).max(), np.abs(Fy).max())
    worst = 0.0
    for i in cells:
        for comp in (0, 1):
            xp, yp, xm, ym = x.copy(), y.copy(), x.copy(), y.copy()
            if comp == 0:
                xp[i] += h
                xm[i] -= h
            else:
                yp[i] += h
                ym[i] -= h
            Ep = oracle.energy(xp, yp, Lx, Ly, topo, p0, A0, KA, KP)
            Em = oracle.energy(xm, ym, Lx, Ly, topo, p0, A0, KA, KP)
            fd = -(Ep - Em) / (2 * h)
            f = Fx[i] if comp == 0 else Fy[i]
            worst = max(worst, abs(fd - f) / scale)
    return worst


@pytest.mark.parametrize("p0,A0,KA,KP", [(3.8, 1.0, 1.0, 1.0), (3.6, 1.3, 0.7, 2.0), (4.1, 0.9, 0.0, 1.0),
                                         (3.9, 1.0, 1.0, 0.0)])
def test_forces_match_finite_differences(p0, A0, KA, KP):
    x, y, th, Lx, Ly = state(100, 5)
    topo = oracle.triangulate(x, y, Lx, Ly)
    assert fd_check(x, y, Lx, Ly, topo, p0, A0, KA, KP, range(0, 100, 9)) < 1e-6


def test_forces_match_fd_with_per_cell_p0():
    x, y, th, Lx, Ly = state(64, 8)
    topo = oracle.triangulate(x, y, Lx, Ly)
    p0 = np.random.default_rng(1).uniform(3.7, 3.9, 64)
    assert fd_check(x, y, Lx, Ly, topo, p0, 1.0, 1.0, 1.0, range(0, 64, 5)) < 1e-6


def test_net_force_vanishes():
    x, y, th, Lx, Ly = state(400, 9)
    topo = oracle.triangulate(x, y, Lx, Ly)
    Fx, Fy, *_ = oracle.forces(x, y, Lx, Ly, topo, 3.85)
    scale = np.abs(Fx).max()
    # translation invariance of E: sum_i F_i = 0
    assert abs(Fx.sum()) < 1e-11 * scale * len(x) and abs(Fy.sum()) < 1e-11 * scale * len(x)


def test_free_active_brownian_particles():
    """K_A = K_P = 0: no forces, so each cell is a free active Brownian
    particle.  For the discrete update with Gaussian director increments the
    mean squared displacement after K steps is exactly
        v0^2 dt^2 sum_{s,s'} exp(-Dr dt |s - s'|),
    and <cos(theta_K - theta_0)> = exp(-Dr dt K)."""
    n, K, dt, Dr, v0 = 1024, 60, 0.02, 1.0, 0.5
    x, y, th, Lx, Ly = state(n, 21)
    x1, y1, th1, _ = oracle.spv_run(x, y, th, Lx, Ly, 3.8, v0, K, seed=99, KA=0.0, KP=0.0, Dr=Dr,
                                    dt=dt)
    dx = (x1 - x + Lx / 2) % Lx - Lx / 2
    dy = (y1 - y + Ly / 2) % Ly - Ly / 2
    r2 = dx * dx + dy * dy
    s = np.arange(K)
    theory = v0 ** 2 * dt ** 2 * np.exp(-Dr * dt * np.abs(s[:, None] - s[None, :])).sum()
    se = r2.std() / math.sqrt(n)
    assert abs(r2.mean() - theory) < 4 * se
    c = np.cos(th1 - th)
    assert abs(c.mean() - math.exp(-Dr * dt * K)) < 4 * c.std() / math.sqrt(n)


def test_gradient_descent_lowers_energy():
    """v0 = 0 and D_r = 0 reduce Eq. 3 to gradient descent dr/dt = -mu grad E:
    at small dt the energy must not increase."""
    x, y, th, Lx, Ly = state(200, 4)
    energies = []
    for step in range(8):
        topo = oracle.triangulate(x, y, Lx, Ly)
        energies.append(oracle.energy(x, y, Lx, Ly, topo, 3.7))
        x, y, th, _ = oracle.spv_run(x, y, th, Lx, Ly, 3.7, 0.0, 1, seed=1, step0=step, Dr=0.0,
                                     dt=0.01)
    assert all(b < a for a, b in zip(energies, energies[1:]))


def test_single_step_update_formula():
    """Eq. 3, one Euler-Maruyama step, with forces from the oracle."""
    x, y, th, Lx, Ly = state(64, 6)
    topo = oracle.triangulate(x, y, Lx, Ly)
    Fx, Fy, *_ = oracle.forces(x, y, Lx, Ly, topo, 3.8)
    x1, y1, th1 = oracle.integrate(x, y, th, Fx, Fy, Lx, Ly, 0.1, 1.0, 1.0, 0.01, 5, 3)
    q = oracle.grid_exponent(Lx, Ly)
    ex = (x + 0.01 * (Fx + 0.1 * np.cos(th))) % Lx
    ey = (y + 0.01 * (Fy + 0.1 * np.sin(th))) % Ly
    dxm = (x1 - ex + Lx / 2) % Lx - Lx / 2
    dym = (y1 - ey + Ly / 2) % Ly - Ly / 2
    # snapping moves a position by at most half a grid unit
    assert np.abs(dxm).max() <= 2.0 ** (-q) and np.abs(dym).max() <= 2.0 ** (-q)
    xi = np.array([oracle.director_noise(5, i, 3) for i in range(64)])
    np.testing.assert_allclose(th1, th + math.sqrt(2 * 1.0 * 0.01) * xi, rtol=0, atol=1e-15)


def test_update_with_a_tag_offset():
    """Eq. 3 for a system whose cells carry noise counters tag0 + i (a
    replica placed after others in a batch): positions as without the offset,
    directors rotated by the noise of counters tag0 + i."""
    x, y, th, Lx, Ly = state(64, 7)
    topo = oracle.triangulate(x, y, Lx, Ly)
    Fx, Fy, *_ = oracle.forces(x, y, Lx, Ly, topo, 3.8)
    x0, y0, th0 = oracle.integrate(x, y, th, Fx, Fy, Lx, Ly, 0.1, 1.0, 1.0, 0.01, 5, 3)
    x1, y1, th1 = oracle.integrate(x, y, th, Fx, Fy, Lx, Ly, 0.1, 1.0, 1.0, 0.01, 5, 3, tag0=1000)
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(y1, y0)
    xi = np.array([oracle.director_noise(5, 1000 + i, 3) for i in range(64)])
    np.testing.assert_allclose(th1, th + math.sqrt(2 * 1.0 * 0.01) * xi, rtol=0, atol=1e-15)
    assert np.abs(th1 - th0).max() > 1e-3


def test_window_step_equals_full_step():
    """The spatial-window step used to time bounded samples of a large
    workload reproduces the full periodic step exactly for its interior cells."""
    x, y, th, Lx, Ly = state(4096, 13)
    x1, y1, th1, _ = oracle.spv_run(x, y, th, Lx, Ly, 3.85, 0.1, 1, seed=5, step0=2)
    wx, wy, wth, k = oracle.spv_window_step(x, y, th, Lx, Ly, 3.85, 0.1, 5, 2, 32.0, 32.0, 12.0)
    upd = np.nonzero((wx != x) | (wy != y) | (wth != th))[0]
    assert k > 400 and len(upd) == k
    np.testing.assert_array_equal(wx[upd], x1[upd])
    np.testing.assert_array_equal(wy[upd], y1[upd])
    np.testing.assert_array_equal(wth[upd], th1[upd])
