"""Host logic of the strip decomposition (paper_1702_02939_gb300.domains) on CPU.

A domain-decomposed run must reproduce the undivided run exactly for the cells
each domain owns (the paper names domain decomposition as the way to larger
systems, Sec. 4; forces reach the next-nearest neighbours, App. A.2, hence the
halos).  The partition, the halo lists, the exchange, the gather and the
re-partition (migration) are host code; here they drive a small stand-in
engine written for the test -- short-range pair forces evaluated by brute
force in each domain's periodic frame, integer-exact moves on the position
grid, the same pending-position semantics as the library's contexts -- so that
the whole protocol runs on CPU, in one process and over two gloo ranks, and is
checked bit for bit against the same engine on the undivided box.  The GPU
engine (the library's contexts) is checked the same way in
tests/test_gpu_domains.py.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1702_02939_gb300 import domains  # noqa: E402

RC = 1.6     # pair cutoff of the stand-in engine (box units)
DT = 0.004


class PairEngine:
    """Stand-in engine: x' = x + round(dt F 2^q) with F_i the sum, over the
    cells within RC in increasing global index, of a smooth repulsion; the
    box is the domain's frame, periodic (its seam is wrong by design, as a
    library context's is, and only halo cells near it see that)."""

    def __init__(self, part, d, x, y, theta, ids, step, p0, v0, frame=True):
        self.part = part
        if frame:
            X0, width = part.frame(d)
        else:
            X0, width = 0, part.LX
        self.X0, self.width = X0, width
        self.ids = ids
        self.cur = np.stack([np.mod(part.grid(x) - X0, part.LX), np.mod(part.grid(y), part.LY)])
        assert (self.cur[0] < width).all()
        self.pending = self._move(self.cur)
        self.device = torch.device("cpu")

    def _move(self, P):
        s = self.part.scale
        dx = P[0][None, :] - P[0][:, None]
        dy = P[1][None, :] - P[1][:, None]
        dx = (dx + self.width // 2) % self.width - self.width // 2
        dy = (dy + self.part.LY // 2) % self.part.LY - self.part.LY // 2
        fx, fy = dx / s, dy / s
        r2 = fx * fx + fy * fy
        w = np.where((r2 > 0) & (r2 < RC * RC), (RC * RC - r2) ** 2, 0.0)
        # sums in increasing global index (columns are in that order)
        Fx = -np.sum(w * fx, axis=1)
        Fy = -np.sum(w * fy, axis=1)
        X = np.mod(P[0] + np.rint(DT * Fx * s).astype(np.int64), self.width)
        Y = np.mod(P[1] + np.rint(DT * Fy * s).astype(np.int64), self.part.LY)
        return np.stack([X, Y])

    def slots(self, where, count):
        s = torch.full((len(self.ids),), -1, dtype=torch.int32)
        s[torch.as_tensor(where, dtype=torch.long)] = torch.arange(count, dtype=torch.int32)
        return s

    def buffer(self, count):
        return torch.empty(2 * count, dtype=torch.int64)

    def step(self, k=1):
        for _ in range(k):
            self.cur = self.pending
            self.pending = self._move(self.cur)

    def pack(self, slot, out):
        sl = slot.numpy()
        k = np.nonzero(sl >= 0)[0]
        X = np.mod(self.pending[0, k] + self.X0, self.part.LX)
        out.view(-1, 2)[sl[k], 0] = torch.from_numpy(X)
        out.view(-1, 2)[sl[k], 1] = torch.from_numpy(self.pending[1, k].copy())

    def unpack(self, slot, inp):
        sl = slot.numpy()
        k = np.nonzero(sl >= 0)[0]
        v = inp.view(-1, 2).numpy()[sl[k]]
        X = np.mod(v[:, 0] - self.X0, self.part.LX)
        assert (X < self.width).all(), "halo cell left the frame"
        self.pending = self.pending.copy()
        self.pending[0, k] = X
        self.pending[1, k] = v[:, 1]

    def state(self):
        s = self.part.scale
        x = np.mod(self.cur[0] + self.X0, self.part.LX) / s
        return x, self.cur[1] / s, np.zeros(len(self.ids))

    def close(self):
        pass


def workload(n, seed):
    L = float(np.sqrt(n))
    rng = np.random.default_rng(seed)
    part = domains.StripPartition(L, L, 2, 3.0)
    x = part.grid(rng.uniform(0, L, n)) / part.scale
    y = np.mod(np.rint(rng.uniform(0, L, n) * part.scale), part.LY) / part.scale
    return x, y, np.zeros(n), L


def reference(x, y, L, steps):
    part = domains.StripPartition(L, L, 2, 3.0)
    eng = PairEngine(part, 0, x, y, None, np.arange(len(x)), 0, 0, 0, frame=False)
    eng.step(steps)
    return eng.state()


def test_partition_owns_every_cell_once_and_lists_the_halos():
    n = 1000
    x, y, th, L = workload(n, 3)
    for D in (2, 3, 4):
        part = domains.StripPartition(L, L, D, 3.0)
        plans = part.plan(x)
        owned = np.concatenate([p["ids"][p["owned"]] for p in plans])
        assert np.array_equal(np.sort(owned), np.arange(n))
        X = part.grid(x)
        for d, p in enumerate(plans):
            assert np.all(np.diff(p["ids"]) > 0)  # increasing global index
            # the context holds exactly the cells of its frame less the margins
            X0, width = part.frame(d)
            r = np.mod(X - X0, part.LX)
            assert np.array_equal(p["ids"], np.nonzero((r >= part.M) & (r < width - part.M))[0])
            # every halo cell comes from its owner's send list, once
            halo = p["ids"][~p["owned"]]
            sent = np.concatenate([plans[e]["sends"][d] for e in range(D) if e != d])
            assert np.array_equal(np.sort(sent), halo)
            # a strip's own cells lie in it; the halo reaches W beyond both sides
            lo, hi = part.bounds[d], part.bounds[d + 1]
            assert np.all((X[p["ids"][p["owned"]]] >= lo) & (X[p["ids"][p["owned"]]] < hi))


def test_partition_refuses_halos_that_cover_the_box():
    with pytest.raises(ValueError):
        domains.StripPartition(20.0, 20.0, 2, 6.0)
    with pytest.raises(ValueError):
        domains.StripPartition(20.0, 20.0, 1, 1.0)


@pytest.mark.parametrize("D,every", [(2, 4), (3, 5)])
def test_local_domains_reproduce_the_undivided_run(D, every):
    n, steps = 900, 13
    x, y, th, L = workload(n, 5)
    rx, ry, _ = reference(x, y, L, steps)
    dd = domains.DecomposedSPV(x, y, th, L, L, D, halo=3.0, repartition_every=every,
                               engine=lambda part, d, xx, yy, tt, ids, step, pp, vv:
                               PairEngine(part, d, xx, yy, tt, ids, step, pp, vv))
    dd.step(steps)
    gx, gy, _ = dd.state()
    assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
    # cells moved across strip boundaries: the re-partitions migrated them
    part = dd.part
    assert not np.array_equal(part.owner(part.grid(x)), part.owner(part.grid(gx)))
    dd.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, steps, results):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1702_02939_gb300 import domains as dm

    x, y, th, L = workload(n, 7)
    dd = dm.DecomposedSPV(x, y, th, L, L, world, halo=3.0, repartition_every=4, transport=dm.DistTransport(),
                          engine=lambda part, d, xx, yy, tt, ids, step, pp, vv:
                          PairEngine(part, d, xx, yy, tt, ids, step, pp, vv))
    dd.step(steps)
    gx, gy, _ = dd.state()
    results.put((rank, gx, gy, len(dd.engines), sorted(dd.lists)))
    dd.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_undivided_run():
    """One domain per rank, halo messages over gloo, re-partitions through an
    all-gather: both ranks end with the undivided run's state, bit for bit."""
    world, n, steps = 2, 900, 10
    x, y, th, L = workload(n, 7)
    rx, ry, _ = reference(x, y, L, steps)
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, steps, results)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((results.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gx, gy, neng, keys in out:
        assert neng == 1  # one domain per rank
        assert set(keys) == {(0, 1), (1, 0)}
        assert np.array_equal(gx, rx) and np.array_equal(gy, ry)
