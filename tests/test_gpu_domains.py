"""GPU strip decomposition of one SPV system against the undivided system.

A domain's context holds its strip's cells and a halo (forces reach the
next-nearest neighbours, App. A.2, after Eq. A7); with its box framed in the
large box (cg_set_frame), the cells' global indices as noise counters
(cg_set_noise_ids) and the halo positions replaced from their owners before
every step (cg_halo_pack / cg_halo_unpack), every cell must evolve exactly as
in one context over the whole box (Eq. 3 rounded identically; the same
Delaunay rings), through re-partitions that migrate cells between strips.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1702_02939_gb300 as cg  # noqa: E402
from paper_1702_02939_gb300 import domains  # noqa: E402


def on_grid(x, L):
    q = domains.grid_exponent(L, L)
    s = 2.0 ** q
    return np.mod(np.rint(np.asarray(x) * s), np.rint(L * s)) / s


@pytest.mark.parametrize("D,steps,every", [(2, 60, 25), (3, 40, 15)])
def test_decomposed_run_equals_the_undivided_run(D, steps, every):
    n = 4096
    x, y, th, L = workloads.spv_uniform(n, 61)
    ref = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.85, v0=0.3)], x, y, th, dt=0.01, seed=5)
    # the random start holds nearly coincident cells whose first moves are
    # long: the decomposed run starts from the state after 20 steps
    ref.step(20)
    x, y, th = (t.cpu().numpy() for t in ref.state())
    dd = domains.DecomposedSPV(x, y, th, L, L, D, halo=8.0, p0=3.85, v0=0.3, repartition_every=every,
                               step0=20, dt=0.01, seed=5)
    ref.step(steps)
    dd.step(steps)
    rx, ry, rth = (t.cpu().numpy() for t in ref.state())
    gx, gy, gth = dd.state()
    assert np.array_equal(gx, rx) and np.array_equal(gy, ry) and np.array_equal(gth, rth)
    # the own cells' rings, as global indices, are the undivided system's rings
    cnt, nbr = (t.cpu().numpy() for t in ref.neighbors())
    rings = dd.owned_neighbors()
    assert len(rings) == n
    for i, ring in rings.items():
        assert np.array_equal(ring, nbr[i, :cnt[i]])
    # cells crossed strip boundaries and were migrated by the re-partitions
    part = dd.part
    assert (part.owner(part.grid(x)) != part.owner(part.grid(gx))).any()
    ref.close()
    dd.close()


def test_halo_exchange_refuses_a_position_outside_the_frame():
    n = 1024
    x, y, th, L = workloads.spv_uniform(n, 62)
    x, y = on_grid(x, L), on_grid(y, L)
    sim = cg.SPV([dict(n=n, Lx=L / 2, Ly=L, p0=3.85, v0=0.1)], np.mod(x, L / 2), y, th)
    sim.set_frame(0.0, 0.0, L, L)
    slot = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    slot[5] = 0
    q = domains.grid_exponent(L, L)
    bad = torch.tensor([int(0.75 * L * 2 ** q), 0], dtype=torch.int64, device="cuda")  # x = 3L/4: outside
    sim.halo_unpack(slot, bad)
    with pytest.raises(cg.CellgbError):
        sim.sync()
    sim.close()
    # frames that do not share the position grid, or lie outside the box, are refused
    sim = cg.SPV([dict(n=n, Lx=L / 2, Ly=L, p0=3.85, v0=0.1)], np.mod(x, L / 2), y, th)
    with pytest.raises(cg.CellgbError):
        sim.set_frame(0.0, 0.0, 4 * L, 4 * L)
    with pytest.raises(cg.CellgbError):
        sim.set_frame(1.5 * L, 0.0, L, L)
    sim.close()
