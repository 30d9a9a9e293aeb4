"""Strip decomposition of one large periodic SPV system (host side).

The paper names domain decomposition as the way past one GPU's capacity
(Sec. 4, "Discussion"); the force on a cell reaches its next-nearest
neighbours (App. A.2, the remark after Eq. A7), so a domain also holds a halo
of the cells around the cells it owns.  This module owns the partition of the
box into strips, the halo lists, the per-step exchange of halo positions and
the periodic re-partition that migrates cells whose positions crossed into
another strip.  Every step of the physics runs in the library's kernels, one
context per domain (`SPVEngine`): its box is the frame of the strip plus its
halo inside the large box (cg_set_frame), its cells are passed in increasing
global index with their global indices as noise counters (cg_set_noise_ids),
and the halo cells' pending positions are replaced from their owners before
every step (cg_halo_pack / cg_halo_unpack).  A domain's own cells then evolve
exactly as in the undivided system, bit for bit.

Layout per domain d: the strip [b_d, b_{d+1}) of the x axis (grid units,
b_d = round(d LX / D)), widened by the halo W on both sides into a frame of
width b_{d+1} - b_d + 2 W with origin b_d - W (periodic).  The cells whose x
lies in the frame make up the domain's context: its own cells (x in the
strip) and halo cells (owned by the neighbouring strips).  Between
re-partitions the membership is fixed; halo widths are chosen so that cells
drift far less than the margin in that time.

Transports: `LocalTransport` runs every domain in one process (all contexts
on one CUDA stream, so packing, copying and unpacking are ordered by the
stream); `DistTransport` runs one domain per rank of a torch.distributed
process group (point-to-point messages; with the gloo backend the int64
buffers go through host memory).
"""
import math

import numpy as np

from . import SPV


def grid_exponent(Lx, Ly):
    """q of the position grid 2^-q: 50 - ceil(log2(max side)), as the library."""
    m, e = math.frexp(max(Lx, Ly))
    return 50 - (e - 1 if m == 0.5 else e)


class StripPartition:
    """D strips along x of the periodic box (Lx, Ly), halo `halo` (box units).

    The frame of a strip reaches `halo` beyond both of its sides; the cells of
    the outer `margin` of that band are left out of the domain, so that halo
    cells can drift up to `margin` outwards between re-partitions and stay in
    the frame (default halo / 4)."""

    def __init__(self, Lx, Ly, D, halo, margin=None):
        self.q = grid_exponent(Lx, Ly)
        self.scale = 2.0 ** self.q
        self.LX = int(round(Lx * self.scale))
        self.LY = int(round(Ly * self.scale))
        self.Lx = self.LX / self.scale
        self.Ly = self.LY / self.scale
        self.D = int(D)
        self.W = int(math.ceil(halo * self.scale))
        self.M = int(math.ceil((0.25 * halo if margin is None else margin) * self.scale))
        if not 0 <= self.M < self.W:
            raise ValueError("the margin must be smaller than the halo")
        self.bounds = [int(round(d * self.LX / self.D)) for d in range(self.D + 1)]
        width = max(self.bounds[d + 1] - self.bounds[d] for d in range(self.D))
        if self.D < 2 or width + 2 * self.W >= self.LX:
            raise ValueError("a strip plus its two halos must be narrower than the box (D >= 2)")
        narrow = min(self.bounds[d + 1] - self.bounds[d] for d in range(self.D)) + 2 * self.W
        if grid_exponent(narrow / self.scale, self.Ly) != self.q:
            raise ValueError("the frames must share the box's position grid: cut the strips across the "
                             "longer side (max(frame sides) must round up to the same power of two)")

    def grid(self, x):
        """Grid coordinates of positions that lie on the grid (exact)."""
        X = np.rint(np.asarray(x, np.float64) * self.scale).astype(np.int64)
        return np.mod(X, self.LX)

    def owner(self, X):
        return np.searchsorted(np.asarray(self.bounds[1:-1]), X, side="right")

    def frame(self, d):
        """(origin X0, width) of domain d's frame in grid units."""
        X0 = (self.bounds[d] - self.W) % self.LX
        return X0, self.bounds[d + 1] - self.bounds[d] + 2 * self.W

    def in_frame(self, X, d):
        X0, width = self.frame(d)
        return np.mod(X - X0, self.LX) < width

    def members(self, X, d):
        """Cells of domain d's context: its frame less the outer margins."""
        X0, width = self.frame(d)
        r = np.mod(X - X0, self.LX)
        return (r >= self.M) & (r < width - self.M)

    def plan(self, x):
        """Per domain: the global indices of its context's cells (increasing),
        the mask of the ones it owns, and the send lists to every other domain
        (global indices, increasing: the message order)."""
        X = self.grid(x)
        own = self.owner(X)
        members = [np.nonzero(self.members(X, d))[0] for d in range(self.D)]
        plans = []
        for d in range(self.D):
            ids = members[d]
            sends = {}
            for e in range(self.D):
                if e != d:
                    m = members[e]
                    sends[e] = m[own[m] == d]
            plans.append({"ids": ids, "owned": own[ids] == d, "sends": sends})
        return plans


class SPVEngine:
    """One domain: a library context over the frame of a strip."""

    def __init__(self, part, d, x, y, theta, ids, step, p0, v0, device, **params):
        import torch

        self.torch = torch
        X0, width = part.frame(d)
        self.x0 = X0 / part.scale
        self.Lx_frame = width / part.scale
        # frame coordinates (exact: grid values, reduced modulo the large box)
        xf = np.mod(part.grid(x) - X0, part.LX) / part.scale
        self.sim = SPV([dict(n=len(ids), Lx=self.Lx_frame, Ly=part.Ly, p0=float(np.mean(p0)), v0=float(np.mean(v0)))],
                       xf, y, theta, device=device, **params)
        self.sim.set_noise_ids(ids.astype(np.int32))
        self.sim.set_frame(self.x0, 0.0, part.Lx, part.Ly)
        if np.ndim(p0):
            self.sim.set_p0(p0)
        if np.ndim(v0):
            self.sim.set_v0(v0)
        self.sim.set_step(step)
        self.part = part
        self.device = self.sim.device

    def slots(self, where, count):
        """Slot array (device int32, user order): where[k] = local index of
        message entry k."""
        t = self.torch
        s = t.full((self.sim.n,), -1, dtype=t.int32)
        s[t.as_tensor(where, dtype=t.long)] = t.arange(count, dtype=t.int32)
        return s.to(self.device)

    def buffer(self, count):
        return self.torch.empty(2 * count, dtype=self.torch.int64, device=self.device)

    def step(self, k=1):
        self.sim.step(k)

    def pack(self, slot, out):
        self.sim.halo_pack(slot, out)

    def unpack(self, slot, inp):
        self.sim.halo_unpack(slot, inp)

    def state(self):
        """(x, y, theta) of the context's cells (large-box coordinates), host."""
        self.sim.sync()
        xf, y, th = (t.cpu().numpy() for t in self.sim.state())
        x = np.mod(np.rint(xf * self.part.scale).astype(np.int64) + int(round(self.x0 * self.part.scale)),
                   self.part.LX) / self.part.scale
        return x, y, th

    def neighbors(self):
        cnt, nbr = self.sim.neighbors()
        return cnt.cpu().numpy(), nbr.cpu().numpy()

    def forces(self):
        Fx, Fy, _ = self.sim.forces()
        return Fx.cpu().numpy(), Fy.cpu().numpy()

    def close(self):
        self.sim.close()


class LocalTransport:
    """All domains in this process."""

    def __init__(self, D):
        self.D = D
        self.mine = list(range(D))

    def exchange(self, engines, lists):
        # every context runs on the same stream: the packs follow the steps,
        # the unpacks the packs
        for (d, e), (send_slot, recv_slot, buf) in lists.items():
            engines[d].pack(send_slot, buf)
        for (d, e), (send_slot, recv_slot, buf) in lists.items():
            engines[e].unpack(recv_slot, buf)

    def gather(self, items):
        """items: {domain: value} of this process -> list of such dicts."""
        return [items]


class DistTransport:
    """One domain per rank of the default torch.distributed group."""

    def __init__(self):
        import torch.distributed as dist

        self.dist = dist
        self.D = dist.get_world_size()
        self.rank = dist.get_rank()
        self.mine = [self.rank]
        self.host_staged = dist.get_backend() == "gloo"

    def exchange(self, engines, lists):
        dist = self.dist
        me = self.rank
        eng = engines[me]
        ops, recvs = [], []
        for (d, e), (send_slot, recv_slot, buf) in lists.items():
            if d == me:
                eng.pack(send_slot, buf)
        if self.host_staged and eng.device.type == "cuda":
            eng.torch.cuda.synchronize()
        for (d, e), (send_slot, recv_slot, buf) in sorted(lists.items()):
            if d == me:
                b = buf.cpu() if self.host_staged else buf
                ops.append(dist.P2POp(dist.isend, b, e))
            elif e == me:
                b = buf.new_empty(buf.shape, device="cpu") if self.host_staged else buf
                ops.append(dist.P2POp(dist.irecv, b, d))
                recvs.append((recv_slot, buf, b))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for recv_slot, buf, b in recvs:
            if b is not buf:
                buf.copy_(b)
            eng.unpack(recv_slot, buf)

    def gather(self, items):
        """items: {domain: value} of this rank -> list of every rank's dict."""
        out = [None] * self.D
        self.dist.all_gather_object(out, items)
        return out


class DecomposedSPV:
    """One periodic SPV system of n cells advanced as D strip domains.

    x, y, theta: the whole system (host arrays, positions on the position grid
    of the box, e.g. from oracle-independent snapping by the library's own
    rule: round(x 2^q) 2^-q).  p0, v0: scalars or per-cell arrays.  halo: in
    box units; repartition_every: steps between re-partitions (migration).
    engine: callable (part, d, x, y, theta, ids, step, p0, v0) -> engine
    (default: SPVEngine on `device`).  transport: LocalTransport(D) (default)
    or DistTransport() (one domain per rank; D = world size).  margin: see
    StripPartition.  step0: the step counter of the given state (the noise of
    the next step uses it).
    """

    def __init__(self, x, y, theta, Lx, Ly, D, halo, p0=3.85, v0=0.1, repartition_every=50, transport=None,
                 engine=None, device="cuda", margin=None, step0=0, **params):
        self.transport = transport or LocalTransport(D)
        self.part = StripPartition(Lx, Ly, D, halo, margin)
        self.n = len(x)
        self.p0 = p0 if np.ndim(p0) == 0 else np.asarray(p0, np.float64)
        self.v0 = v0 if np.ndim(v0) == 0 else np.asarray(v0, np.float64)
        self.every = int(repartition_every)
        self.step_count = int(step0)
        self.params = params
        self.device = device
        self.make = engine or (lambda part, d, xx, yy, tt, ids, step, pp, vv: SPVEngine(
            part, d, xx, yy, tt, ids, step, pp, vv, device, **params))
        self.engines = {}
        self._build(np.asarray(x, np.float64), np.asarray(y, np.float64), np.asarray(theta, np.float64))

    def _percell(self, v, ids):
        return v if np.ndim(v) == 0 else v[ids]

    def _build(self, x, y, theta):
        for eng in self.engines.values():
            eng.close()
        self.engines = {}
        self.plans = self.part.plan(x)
        for d in self.transport.mine:
            ids = self.plans[d]["ids"]
            self.engines[d] = self.make(self.part, d, x[ids], y[ids], theta[ids], ids, self.step_count,
                                        self._percell(self.p0, ids), self._percell(self.v0, ids))
        # message lists: (sender, receiver) -> (send slots on the sender,
        # receive slots on the receiver, buffer on whichever side holds it)
        self.lists = {}
        for d in range(self.part.D):
            for e, glob in self.plans[d]["sends"].items():
                if len(glob) == 0 or (d not in self.engines and e not in self.engines):
                    continue
                src = np.searchsorted(self.plans[d]["ids"], glob)
                dst = np.searchsorted(self.plans[e]["ids"], glob)
                here = self.engines.get(d) or self.engines.get(e)
                send = self.engines[d].slots(src, len(glob)) if d in self.engines else None
                recv = self.engines[e].slots(dst, len(glob)) if e in self.engines else None
                self.lists[(d, e)] = (send, recv, here.buffer(len(glob)))
        # the halo cells' pending positions from their owners (a new context
        # computed them from its own cells, which near its frame's edges
        # lack neighbours)
        self.transport.exchange(self.engines, self.lists)

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            for eng in self.engines.values():
                eng.step(1)
            self.step_count += 1
            self.transport.exchange(self.engines, self.lists)
            if self.every and self.step_count % self.every == 0:
                self.repartition()

    def _owned_state(self):
        """This process's domains' own cells: (global ids, x, y, theta)."""
        out = {}
        for d, eng in self.engines.items():
            x, y, th = eng.state()
            own = self.plans[d]["owned"]
            out[d] = (self.plans[d]["ids"][own], x[own], y[own], th[own])
        return out

    def state(self):
        """(x, y, theta) of all cells in global index order (every process)."""
        parts = self.transport.gather(self._owned_state())
        x, y, th = np.empty(self.n), np.empty(self.n), np.empty(self.n)
        for chunk in parts:
            for ids, xx, yy, tt in chunk.values():
                x[ids], y[ids], th[ids] = xx, yy, tt
        return x, y, th

    def repartition(self):
        """Migration: every cell goes to the strip its position now lies in,
        and the halos are rebuilt from the new positions."""
        x, y, th = self.state()
        self._build(x, y, th)

    def owned_neighbors(self):
        """{global id: ring as global ids} of this process's own cells."""
        out = {}
        for d, eng in self.engines.items():
            cnt, nbr = eng.neighbors()
            ids = self.plans[d]["ids"]
            for k in np.nonzero(self.plans[d]["owned"])[0]:
                out[int(ids[k])] = ids[nbr[k, :cnt[k]]]
        return out

    def close(self):
        for eng in self.engines.values():
            eng.close()
        self.engines = {}
