"""GPU backward pass against the oracle adjoint and finite differences.

The reverse pass of Eq. 3 (Sussman, arXiv 1702.02939) with fixed noise needs
Hessian-vector products of E (Eq. 1) through the forces of Eqs. A6-A16; the
library computes them with hand-derived tangent kernels, the oracle with dual
numbers over its own force code.
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


def make(n, iseed, p0=3.8, v0=0.1, **kw):
    x, y, th, L = workloads.spv_uniform(n, iseed)
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    sim = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=p0, v0=v0)], xs, ys, th, **kw)
    return sim, xs, ys, th, Lx, Ly


def shape_loss(A, P, target=3.95):
    r = P * np.sqrt(A) - target * A
    n = len(A)
    return (r * r).mean(), 2.0 * r * (P / (2.0 * np.sqrt(A)) - target) / n, 2.0 * r * np.sqrt(A) / n


@pytest.mark.parametrize("n", [400, 4096])
def test_hvp_matches_oracle(n):
    sim, xs, ys, th, Lx, Ly = make(n, 3)
    topo = oracle.triangulate(xs, ys, Lx, Ly)
    rng = np.random.default_rng(5)
    vx, vy = rng.normal(size=n), rng.normal(size=n)
    Hx, Hy, Ad, Pd = (t.cpu().numpy() for t in sim.hvp(vx, vy))
    oHx, oHy, oAd, oPd = oracle.hvp(xs, ys, Lx, Ly, topo, 3.8, vx, vy)
    scale = max(np.abs(oHx).max(), np.abs(oHy).max())
    assert np.abs(Hx - oHx).max() <= 1e-10 * scale
    assert np.abs(Hy - oHy).max() <= 1e-10 * scale
    assert np.abs(Ad - oAd).max() <= 1e-10 * np.abs(oAd).max()
    assert np.abs(Pd - oPd).max() <= 1e-10 * np.abs(oPd).max()
    sim.close()


@pytest.mark.parametrize("K,every", [(6, 4), (12, 5)])
def test_backward_matches_oracle_adjoint(K, every):
    n, seed = 400, 21
    sim, xs, ys, th, Lx, Ly = make(n, 7, seed=seed, dt=0.01)
    p0 = np.random.default_rng(3).uniform(3.7, 3.9, n)
    sim.set_p0(p0)
    sim.set_step(0)
    bw = sim.run_checkpointed(K, every)
    A, P = (t.cpu().numpy() for t in sim.geometry())
    L, gA, gP = shape_loss(A, P)
    z = np.zeros(n)
    gx0, gy0, gp0, gv0, gKA, gKP = sim.backward(bw, K, every, z, z, gA, gP)
    ref = oracle.spv_backward(xs, ys, th, Lx, Ly, p0, 0.1, K, seed, z, z, gA, gP)
    np.testing.assert_allclose(A, ref["A"], rtol=1e-11)
    gpos = max(np.abs(ref["gx0"]).max(), np.abs(ref["gy0"]).max())
    assert np.abs(gx0.cpu().numpy() - ref["gx0"]).max() <= 1e-9 * gpos
    assert np.abs(gy0.cpu().numpy() - ref["gy0"]).max() <= 1e-9 * gpos
    assert np.abs(gp0.cpu().numpy() - ref["gp0"]).max() <= 1e-9 * np.abs(ref["gp0"]).max()
    assert np.abs(gv0.cpu().numpy() - ref["gv0"]).max() <= 1e-9 * np.abs(ref["gv0"]).max()
    assert abs(gKA - ref["gKA"]) <= 1e-9 * abs(ref["gKA"]) + 1e-12
    assert abs(gKP - ref["gKP"]) <= 1e-9 * abs(ref["gKP"]) + 1e-12
    sim.close()


@pytest.mark.parametrize("h", [1e-6, 1e-5])
def test_autograd_function_matches_finite_differences(h):
    """loss.backward() through the autograd Function equals central finite
    differences of GPU forward runs on a topology-stable window, to 1e-6 of
    the largest gradient component.  At h = 1e-6 the rounding of every move
    to the position grid (2^-q) adds a resolution floor of about half the
    bound; at h = 1e-5 that floor is a twentieth of it and the truncation
    error of the central difference (~h^2) is still far below it."""
    n, K = 256, 5
    sim, xs, ys, th, Lx, Ly = make(n, 9, seed=4, dt=0.01)
    dev = torch.device("cuda")
    x0 = torch.tensor(xs, device=dev, requires_grad=True)
    y0 = torch.tensor(ys, device=dev, requires_grad=True)
    p0 = torch.tensor(np.random.default_rng(1).uniform(3.7, 3.9, n), device=dev, requires_grad=True)
    v0 = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    KA = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    KP = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    th0 = torch.tensor(th, device=dev)

    def loss_of(xx, yy, pp, vv, ka, kp):
        x, y, A, P = cg.spv_run_differentiable(sim, xx, yy, pp, vv, ka, kp, th0, K, ckpt_every=2)
        return ((P * A.sqrt() - 3.95 * A) ** 2).mean(), sim.neighbors()[1].clone()

    L0, nbr0 = loss_of(x0, y0, p0, v0, KA, KP)
    L0.backward()

    def fd(**delta):
        args = dict(xx=x0.detach(), yy=y0.detach(), pp=p0.detach(), vv=v0.detach(), ka=KA.detach(), kp=KP.detach())
        out = []
        for s in (+1, -1):
            a = {k: (v + s * h * delta[k] if k in delta else v) for k, v in args.items()}
            Ls, nbr = loss_of(a["xx"], a["yy"], a["pp"], a["vv"], a["ka"], a["kp"])
            assert torch.equal(nbr, nbr0)  # topology-stable window
            out.append(float(Ls))
        return (out[0] - out[1]) / (2 * h)

    gpos = max(float(x0.grad.abs().max()), float(y0.grad.abs().max()))
    # resolution of a central difference here: round-off ~1e-8 |L|, plus the
    # rounding of every move to the position grid 2^-q (the runs differ by
    # ~h per step, rounded independently): ~ max|dL/dr| 2^-q sqrt(n K) / h
    q = oracle.grid_exponent(Lx, Ly)
    floor = 1e-8 * abs(float(L0.detach())) + gpos * 2.0 ** (-q) * np.sqrt(n * K) / h
    for i in (0, 100, 200):
        e = torch.zeros(n, dtype=torch.float64, device=dev)
        e[i] = 1.0
        assert abs(fd(xx=e) - float(x0.grad[i])) <= 1e-6 * gpos + floor
        assert abs(fd(yy=e) - float(y0.grad[i])) <= 1e-6 * gpos + floor
        assert abs(fd(pp=e) - float(p0.grad[i])) <= 1e-6 * float(p0.grad.abs().max()) + floor
    one = torch.tensor(1.0, dtype=torch.float64)
    assert abs(fd(vv=one) - float(v0.grad)) <= 1e-6 * abs(float(v0.grad)) + floor
    assert abs(fd(ka=one) - float(KA.grad)) <= 1e-6 * abs(float(KA.grad)) + floor
    assert abs(fd(kp=one) - float(KP.grad)) <= 1e-6 * abs(float(KP.grad)) + floor
    sim.close()
