"""The allocation-free triangulation entry point.

Callers that cannot allocate device memory (fixed memory pools, allocator or
plugin hooks of other runtimes, fully pre-reserved devices) triangulate through
cg_triangulate_noalloc, whose scratch is a static array inside the library.
Its output must equal the regular path's (cg_create + cg_get_neighbors) bit for
bit, on two calls in a row (the second call reuses the array the first one
left behind).  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1702_02939_gb300 as cg  # noqa: E402


def regular_rings(x, y, Lx, Ly=None):
    Ly = Lx if Ly is None else Ly
    sim = cg.SPV([dict(n=len(x), Lx=Lx, Ly=Ly, p0=3.8, v0=0.0)], x, y, np.zeros(len(x)))
    cnt, nbr = sim.neighbors()
    out = cnt.cpu().numpy(), nbr.cpu().numpy()
    sim.close()
    return out


def noalloc_rings(x, y, Lx, Ly=None):
    Ly = Lx if Ly is None else Ly
    n = len(x)
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy = torch.tensor(y, dtype=torch.float64, device="cuda")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda")
    nbr = torch.empty(n * cg.MAX_RING, dtype=torch.int32, device="cuda")
    cg.cg_triangulate_noalloc(n, Lx, Ly, dx, dy, cnt, nbr, torch.cuda.current_stream().cuda_stream)
    return cnt.cpu().numpy(), nbr.view(n, cg.MAX_RING).cpu().numpy()


def raw_call(n, Lx, Ly, x, y):
    """Status of the C entry point itself, on valid device buffers of n
    cells (outputs zero-filled beforehand)."""
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy = torch.tensor(y, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    nbr = torch.zeros(n * cg.MAX_RING, dtype=torch.int32, device="cuda")
    rc = cg.lib().cg_triangulate_noalloc(n, Lx, Ly, cg._ptr(dx), cg._ptr(dy), cg._ptr(cnt), cg._ptr(nbr), None)
    torch.cuda.synchronize()
    return rc, cnt


def test_noalloc_matches_regular_path_twice():
    cases = [workloads.spv_uniform(4096, 31), workloads.spv_uniform(1000, 32)]
    for x, y, th, L in cases:
        c0, n0 = regular_rings(x, y, L)
        c1, n1 = noalloc_rings(x, y, L)
        np.testing.assert_array_equal(c1, c0)
        np.testing.assert_array_equal(n1, n0)
        assert int(c1.sum()) == 6 * len(x)


def test_noalloc_rejects_oversize():
    n = cg.NOALLOC_MAX_CELLS + 1
    x, y, th, L = workloads.spv_uniform(n, 3)
    with pytest.raises(cg.CellgbError):
        noalloc_rings(x, y, L)
    # the C entry point itself refuses the size, with valid device buffers
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy = torch.tensor(y, dtype=torch.float64, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    nbr = torch.zeros(n * cg.MAX_RING, dtype=torch.int32, device="cuda")
    rc = cg.lib().cg_triangulate_noalloc(n, L, L, cg._ptr(dx), cg._ptr(dy), cg._ptr(cnt), cg._ptr(nbr), None)
    assert rc == -1
    assert int(cnt.abs().sum()) == 0  # nothing was written


def test_noalloc_rectangular_box_matches_regular_path():
    # a 2:1 box that fits the bin limit, compared bit for bit
    n, Lx, Ly = 2048, 64.0, 32.0
    x, y, th = workloads.spv_uniform_rect(n, 33, Lx, Ly)
    c0, n0 = regular_rings(x, y, Lx, Ly)
    c1, n1 = noalloc_rings(x, y, Lx, Ly)
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(n1, n0)


def test_noalloc_rejects_bad_inputs():
    # fewer than 16 cells: refused before any GPU work
    x, y, th, L = workloads.spv_uniform(15, 4)
    rc, cnt = raw_call(15, L, L, x, y)
    assert rc == -1 and int(cnt.abs().sum()) == 0
    # a thin box whose cell list would need more than 4 * CG_NOALLOC_MAX_CELLS
    # bins: refused before any GPU work
    n, Lx, Ly = cg.NOALLOC_MAX_CELLS, 2.0, float(cg.NOALLOC_MAX_CELLS) / 2.0
    x, y, th = workloads.spv_uniform_rect(n, 5, Lx, Ly)
    rc, cnt = raw_call(n, Lx, Ly, x, y)
    assert rc == -1 and int(cnt.abs().sum()) == 0
    # one position outside [-L, 2L): the device-side input check refuses it
    x, y, th, L = workloads.spv_uniform(1024, 6)
    x = x.copy()
    x[17] = 2.0 * L
    rc, _ = raw_call(1024, L, L, x, y)
    assert rc == -1
    # the array is left usable: a valid call right after still matches
    x, y, th, L = workloads.spv_uniform(1024, 7)
    c0, n0 = regular_rings(x, y, L)
    c1, n1 = noalloc_rings(x, y, L)
    np.testing.assert_array_equal(c1, c0)
    np.testing.assert_array_equal(n1, n0)
