"""CPU oracle for the cellGPU SPV/AVM hot path (Sussman, arXiv 1702.02939).

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-correct C++ restatement of
the method, loaded with ctypes.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import it; the library never does.  It
shares no code with the CUDA path.
"""
import ctypes as C
import numpy as np

from . import build as _build

MAX_RING = 16
_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)
_up = C.POINTER(C.c_uint32)


def _declare(L):
    L.cgo_grid_exponent.argtypes = [C.c_double, C.c_double]
    L.cgo_grid_exponent.restype = C.c_int
    L.cgo_snap_length.argtypes = [C.c_double, C.c_int]
    L.cgo_snap_length.restype = C.c_double
    L.cgo_snap_positions.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp]
    L.cgo_philox.argtypes = [_up, _up, _up]
    L.cgo_philox.restype = None
    L.cgo_director_noise.argtypes = [C.c_uint64, C.c_int32, C.c_int64]
    L.cgo_director_noise.restype = C.c_double
    L.cgo_orient2d.argtypes = [_lp, _lp, _lp]
    L.cgo_incircle.argtypes = [_lp, _lp, _lp, _lp]
    L.cgo_incircle_sos.argtypes = [_lp, _lp, _lp, _lp, _lp]
    L.cgo_delaunay_plain.argtypes = [C.c_int, _lp, _lp, C.c_int, _ip, _ip]
    L.cgo_triangulate.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_int, _ip, _ip, _ip]
    L.cgo_geometry.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, C.c_int,
                               _dp, _dp, _dp, _dp]
    L.cgo_forces.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, C.c_int,
                             _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.cgo_integrate.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                C.c_uint64, C.c_int64]
    L.cgo_integrate_tagged.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                       C.c_uint64, C.c_int64, C.c_int64]
    L.cgo_spv_run.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp,
                              C.c_uint64, C.c_int64, C.c_int64, _dp, _dp, _dp, _dp]
    L.cgo_spv_window_step.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp,
                                      C.c_uint64, C.c_int64, C.c_double, C.c_double, C.c_double,
                                      C.c_double]
    L.cgo_spv_window_step.restype = C.c_int
    for name in ("cgo_snap_positions", "cgo_orient2d", "cgo_incircle", "cgo_incircle_sos",
                 "cgo_delaunay_plain", "cgo_triangulate", "cgo_geometry", "cgo_forces",
                 "cgo_integrate", "cgo_integrate_tagged", "cgo_spv_run"):
        getattr(L, name).restype = C.c_int
    L.cgo_avm_build.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _ip, _ip, _ip, _ip]
    L.cgo_avm_forces.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, _ip, _dp, _dp,
                                 _dp, _dp, _dp, _dp, _dp, _dp]
    L.cgo_avm_t1.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, _ip, C.c_double,
                             C.c_double, C.c_double, C.c_int, _ip]
    L.cgo_avm_step.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _ip, _ip, _ip, _ip, _dp, _dp,
                               _dp, _dp, C.c_uint64, C.c_int64, C.c_int, _ip]
    L.cgo_avm_divide.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, _ip, _dp, _dp,
                                 _dp, _dp, C.c_int, _ip, _dp, _ip]
    for name in ("cgo_avm_build", "cgo_avm_forces", "cgo_avm_t1", "cgo_avm_step", "cgo_avm_divide"):
        getattr(L, name).restype = C.c_int
    for extra in ("_declare_avm", "_declare_adjoint"):
        fn = globals().get(extra)
        if fn is not None:
            fn(L)


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _l(a):
    return a.ctypes.data_as(_lp)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


def grid_exponent(Lx, Ly):
    return lib().cgo_grid_exponent(float(Lx), float(Ly))


def snap_length(L, q):
    return lib().cgo_snap_length(float(L), int(q))


def box(Lx, Ly=None):
    """Box lengths snapped onto the position grid: (Lx, Ly, q)."""
    Ly = Lx if Ly is None else Ly
    q = grid_exponent(Lx, Ly)
    return snap_length(Lx, q), snap_length(Ly, q), q


def snap_positions(x, y, Lx, Ly):
    x = np.array(x, dtype=np.float64, copy=True)
    y = np.array(y, dtype=np.float64, copy=True)
    _check(lib().cgo_snap_positions(len(x), Lx, Ly, _d(x), _d(y)), "snap")
    return x, y


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().cgo_philox(c, k, o)
    return [int(v) for v in o]


def director_noise(seed, tag, step):
    return lib().cgo_director_noise(int(seed), int(tag), int(step))


def _pt(p):
    return (C.c_int64 * 2)(int(p[0]), int(p[1]))


def orient2d(a, b, c):
    return lib().cgo_orient2d(_pt(a), _pt(b), _pt(c))


def incircle(a, b, c, d):
    return lib().cgo_incircle(_pt(a), _pt(b), _pt(c), _pt(d))


def incircle_sos(a, b, c, d, keys):
    k = (C.c_int64 * 4)(*[int(v) for v in keys])
    return lib().cgo_incircle_sos(_pt(a), _pt(b), _pt(c), _pt(d), k)


def delaunay_plain(X, Y, max_ring=64):
    X = np.ascontiguousarray(X, dtype=np.int64)
    Y = np.ascontiguousarray(Y, dtype=np.int64)
    m = len(X)
    cnt = np.zeros(m, np.int32)
    nbr = np.full(m * max_ring, -1, np.int32)
    _check(lib().cgo_delaunay_plain(m, _l(X), _l(Y), max_ring, _i(cnt), _i(nbr)), "delaunay")
    return cnt, nbr.reshape(m, max_ring)


class Topology:
    """Rings of a periodic Delaunay triangulation: neighbour tags, CCW from the
    smallest tag, with the periodic image offset of each neighbour."""

    def __init__(self, cnt, nbr, off):
        self.cnt, self.nbr, self.off = cnt, nbr, off

    def rings(self):
        return [tuple(int(v) for v in self.nbr[i, :self.cnt[i]]) for i in range(len(self.cnt))]


def triangulate(x, y, Lx, Ly):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = len(x)
    cnt = np.zeros(n, np.int32)
    nbr = np.full(n * MAX_RING, -1, np.int32)
    off = np.zeros(n * MAX_RING * 2, np.int32)
    _check(lib().cgo_triangulate(n, Lx, Ly, _d(x), _d(y), MAX_RING, _i(cnt), _i(nbr), _i(off)),
           "triangulate")
    return Topology(cnt, nbr.reshape(n, MAX_RING), off.reshape(n, MAX_RING, 2))


def geometry(x, y, Lx, Ly, topo):
    n = len(x)
    A = np.zeros(n)
    P = np.zeros(n)
    hx = np.zeros(n * MAX_RING)
    hy = np.zeros(n * MAX_RING)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    _check(lib().cgo_geometry(n, Lx, Ly, _d(x), _d(y), _i(topo.cnt), _i(topo.nbr), _i(topo.off),
                              MAX_RING, _d(A), _d(P), _d(hx), _d(hy)), "geometry")
    return A, P, hx.reshape(n, MAX_RING), hy.reshape(n, MAX_RING)


def forces(x, y, Lx, Ly, topo, p0, A0=1.0, KA=1.0, KP=1.0):
    n = len(x)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    p0 = np.ascontiguousarray(np.broadcast_to(np.asarray(p0, np.float64), (n,)))
    mech = np.array([A0, KA, KP], np.float64)
    Fx, Fy, A, P, E = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(1)
    _check(lib().cgo_forces(n, Lx, Ly, _d(x), _d(y), _i(topo.cnt), _i(topo.nbr), _i(topo.off),
                            MAX_RING, _d(p0), _d(mech), _d(Fx), _d(Fy), _d(A), _d(P), _d(E)),
           "forces")
    return Fx, Fy, A, P, float(E[0])


def energy(x, y, Lx, Ly, topo, p0, A0=1.0, KA=1.0, KP=1.0):
    return forces(x, y, Lx, Ly, topo, p0, A0, KA, KP)[4]


def integrate(x, y, theta, Fx, Fy, Lx, Ly, v0, mu, Dr, dt, seed, step, tag0=0):
    """Eq. 3 for one step from the given forces; the director noise of cell i
    is drawn with counter tag0 + i (tag0 > 0: a system whose cells follow
    others in a larger numbering, as a replica in a batch)."""
    n = len(x)
    x = np.array(x, np.float64, copy=True)
    y = np.array(y, np.float64, copy=True)
    theta = np.array(theta, np.float64, copy=True)
    Fx = np.ascontiguousarray(Fx, dtype=np.float64)
    Fy = np.ascontiguousarray(Fy, dtype=np.float64)
    v0 = np.ascontiguousarray(np.broadcast_to(np.asarray(v0, np.float64), (n,)))
    par = np.array([mu, Dr, dt], np.float64)
    _check(lib().cgo_integrate_tagged(n, Lx, Ly, _d(x), _d(y), _d(theta), _d(Fx), _d(Fy), _d(v0),
                                      _d(par), int(seed), int(step), int(tag0)), "integrate")
    return x, y, theta


def spv_run(x, y, theta, Lx, Ly, p0, v0, nsteps, seed, step0=0, A0=1.0, KA=1.0, KP=1.0, mu=1.0,
            Dr=1.0, dt=0.01):
    """nsteps oracle steps (each retriangulates from scratch). Returns the new
    state and the forces/areas/perimeters evaluated at the last step's start."""
    n = len(x)
    x = np.array(x, np.float64, copy=True)
    y = np.array(y, np.float64, copy=True)
    theta = np.array(theta, np.float64, copy=True)
    p0 = np.ascontiguousarray(np.broadcast_to(np.asarray(p0, np.float64), (n,)))
    v0 = np.ascontiguousarray(np.broadcast_to(np.asarray(v0, np.float64), (n,)))
    par = np.array([A0, KA, KP, mu, Dr, dt], np.float64)
    Fx, Fy, A, P = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib().cgo_spv_run(n, Lx, Ly, _d(x), _d(y), _d(theta), _d(p0), _d(v0), _d(par),
                             int(seed), int(step0), int(nsteps), _d(Fx), _d(Fy), _d(A), _d(P)),
           "spv_run")
    return x, y, theta, (Fx, Fy, A, P)


def spv_window_step(x, y, theta, Lx, Ly, p0, v0, seed, step, cx, cy, hw, margin=6.0, A0=1.0, KA=1.0,
                    KP=1.0, mu=1.0, Dr=1.0, dt=0.01):
    """One oracle step for the cells within hw of (cx, cy) (in place on copies).
    Returns (x, y, theta, number of updated cells)."""
    n = len(x)
    x = np.array(x, np.float64, copy=True)
    y = np.array(y, np.float64, copy=True)
    theta = np.array(theta, np.float64, copy=True)
    p0 = np.ascontiguousarray(np.broadcast_to(np.asarray(p0, np.float64), (n,)))
    v0 = np.ascontiguousarray(np.broadcast_to(np.asarray(v0, np.float64), (n,)))
    par = np.array([A0, KA, KP, mu, Dr, dt], np.float64)
    k = lib().cgo_spv_window_step(n, Lx, Ly, _d(x), _d(y), _d(theta), _d(p0), _d(v0), _d(par), int(seed),
                                  int(step), float(cx), float(cy), float(hw), float(margin))
    if k < 0:
        raise OracleError(f"window step failed with code {k}")
    return x, y, theta, k


def _declare_adjoint(L):
    L.cgo_hvp.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, C.c_int, _dp, _dp, _dp, _dp,
                          _dp, _dp, _dp, _dp]
    L.cgo_hvp.restype = C.c_int
    L.cgo_geom_grad.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _ip, _ip, _ip, C.c_int, _dp, _dp, _dp,
                                _dp]
    L.cgo_geom_grad.restype = C.c_int
    L.cgo_spv_backward.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp, C.c_uint64,
                                   C.c_int64, C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                   _dp, _dp]
    L.cgo_spv_backward.restype = C.c_int


def _f64(a, n):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (n,)))


def hvp(x, y, Lx, Ly, topo, p0, vx, vy, A0=1.0, KA=1.0, KP=1.0):
    """H v (Hessian of E times v) and dA/dv, dP/dv on the given topology."""
    n = len(x)
    x, y, vx, vy, p0 = _f64(x, n), _f64(y, n), _f64(vx, n), _f64(vy, n), _f64(p0, n)
    mech = np.array([A0, KA, KP], np.float64)
    Hx, Hy, Ad, Pd = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib().cgo_hvp(n, Lx, Ly, _d(x), _d(y), _i(topo.cnt), _i(topo.nbr), _i(topo.off), MAX_RING, _d(p0),
                         _d(mech), _d(vx), _d(vy), _d(Hx), _d(Hy), _d(Ad), _d(Pd)), "hvp")
    return Hx, Hy, Ad, Pd


def geom_grad(x, y, Lx, Ly, topo, cA, cP):
    """Gradient of sum_c (cA_c A_c + cP_c P_c) with respect to the positions."""
    n = len(x)
    x, y, cA, cP = _f64(x, n), _f64(y, n), _f64(cA, n), _f64(cP, n)
    gx, gy = np.zeros(n), np.zeros(n)
    _check(lib().cgo_geom_grad(n, Lx, Ly, _d(x), _d(y), _i(topo.cnt), _i(topo.nbr), _i(topo.off), MAX_RING,
                               _d(cA), _d(cP), _d(gx), _d(gy)), "geom_grad")
    return gx, gy


def spv_backward(x0, y0, theta0, Lx, Ly, p0, v0, nsteps, seed, gxT, gyT, gAT, gPT, step0=0, A0=1.0, KA=1.0,
                 KP=1.0, mu=1.0, Dr=1.0, dt=0.01):
    """Forward run plus reverse pass.  Returns dict with the final state
    (x, y, A, P) and the cotangents gx0, gy0, gp0, gv0 (per cell), gKA, gKP."""
    n = len(x0)
    x0, y0, th, p0, v0 = _f64(x0, n), _f64(y0, n), _f64(theta0, n), _f64(p0, n), _f64(v0, n)
    gxT, gyT, gAT, gPT = _f64(gxT, n), _f64(gyT, n), _f64(gAT, n), _f64(gPT, n)
    par = np.array([A0, KA, KP, mu, Dr, dt], np.float64)
    out = {k: np.zeros(n) for k in ("x", "y", "A", "P", "gx0", "gy0", "gp0", "gv0")}
    gK = np.zeros(2)
    _check(lib().cgo_spv_backward(n, Lx, Ly, _d(x0), _d(y0), _d(th), _d(p0), _d(v0), _d(par), int(seed), int(step0),
                                  int(nsteps), _d(gxT), _d(gyT), _d(gAT), _d(gPT), _d(out["x"]), _d(out["y"]),
                                  _d(out["A"]), _d(out["P"]), _d(out["gx0"]), _d(out["gy0"]), _d(out["gp0"]),
                                  _d(out["gv0"]), _d(gK)), "spv_backward")
    out["gKA"], out["gKP"] = float(gK[0]), float(gK[1])
    return out


class AvmNet:
    """Vertex network of the active vertex model: vertex positions (hx, hy),
    per-vertex cells and neighbours (vc, vn: V x 3, CCW, edge v-vn[k] between
    vc[k] and vc[k+1]) and per-cell CCW vertex lists (cc, cv)."""

    def __init__(self, n, Lx, Ly, hx, hy, vc, vn, cc, cv):
        self.n, self.Lx, self.Ly = n, Lx, Ly
        self.hx, self.hy, self.vc, self.vn, self.cc, self.cv = hx, hy, vc, vn, cc, cv

    @property
    def V(self):
        return len(self.hx)

    def copy(self):
        return AvmNet(self.n, self.Lx, self.Ly, *(a.copy() for a in (self.hx, self.hy, self.vc, self.vn, self.cc,
                                                                      self.cv)))

    def _args(self):
        return (self.n, self.V, self.Lx, self.Ly, _d(self.hx), _d(self.hy), _i(self.vc), _i(self.vn), _i(self.cc),
                _i(self.cv))

    def with_capacity(self, cap):
        """The network with `cap` cell slots (2 cap vertex slots): slots past
        the network are empty cells (cc 0, cv -1) and free vertices (-1)."""
        n, V = self.n, self.V
        hx, hy = np.zeros(2 * cap), np.zeros(2 * cap)
        hx[:V], hy[:V] = self.hx, self.hy
        vc, vn = np.full(6 * cap, -1, np.int32), np.full(6 * cap, -1, np.int32)
        vc[:3 * V], vn[:3 * V] = self.vc, self.vn
        cc, cv = np.zeros(cap, np.int32), np.full(cap * MAX_RING, -1, np.int32)
        cc[:n], cv[:n * MAX_RING] = self.cc, self.cv
        return AvmNet(cap, self.Lx, self.Ly, hx, hy, vc, vn, cc, cv)


def avm_build(x, y, Lx, Ly):
    """Voronoi tessellation of the seed positions as a vertex network."""
    n = len(x)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    hx, hy = np.zeros(2 * n), np.zeros(2 * n)
    vc, vn = np.zeros(6 * n, np.int32), np.zeros(6 * n, np.int32)
    cc, cv = np.zeros(n, np.int32), np.full(n * MAX_RING, -1, np.int32)
    _check(lib().cgo_avm_build(n, Lx, Ly, _d(x), _d(y), _d(hx), _d(hy), _i(vc), _i(vn), _i(cc), _i(cv)), "avm_build")
    return AvmNet(n, Lx, Ly, hx, hy, vc, vn, cc, cv)


def _cells(net, v):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (net.n,)))


def avm_forces(net, p0, A0=1.0, KA=1.0, KP=1.0):
    """Vertex forces, areas, perimeters and energy; p0 and A0 scalars or per
    cell (P0_c = p0_c sqrt(A0_c)); removed cells (cc = 0) contribute nothing."""
    p0, a0 = _cells(net, p0), _cells(net, A0)
    mech = np.array([KA, KP], np.float64)
    Fx, Fy, A, P, E = np.zeros(net.V), np.zeros(net.V), np.zeros(net.n), np.zeros(net.n), np.zeros(1)
    _check(lib().cgo_avm_forces(*net._args(), _d(p0), _d(a0), _d(mech), _d(Fx), _d(Fy), _d(A), _d(P), _d(E)),
           "avm_forces")
    return Fx, Fy, A, P, float(E[0])


def avm_transitions(net, thr, newlen=None, t2_area=0.0, cap=16, allow_cap=False):
    """T1 (and, with t2_area > 0, T2) passes on a copy of the network; returns
    (new network, T1s, T2s).  With allow_cap, hitting the pass cap returns
    the partial result."""
    net = net.copy()
    newlen = 1.5 * thr if newlen is None else newlen
    applied = np.zeros(2, np.int32)
    rc = lib().cgo_avm_t1(*net._args(), float(thr), float(newlen), float(t2_area), int(cap), _i(applied))
    if not (allow_cap and rc == -8):
        _check(rc, "avm_t1")
    return net, int(applied[0]), int(applied[1])


def avm_divide(net, cells, dirs, theta, p0, v0, a0):
    """Divisions of cells[k] along dirs[k] = (ux, uy), in order, on copies; each
    one made takes the lowest empty cell slot and the two lowest free vertex
    slots.  Returns (network, theta, p0, v0, a0, made)."""
    net = net.copy()
    theta, p0, v0, a0 = (np.array(a, np.float64, copy=True) for a in (theta, p0, v0, a0))
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1)
    made = np.zeros(len(cells), np.int32)
    _check(lib().cgo_avm_divide(*net._args(), _d(theta), _d(p0), _d(v0), _d(a0), len(cells), _i(cells), _d(dirs),
                                _i(made)), "avm_divide")
    return net, theta, p0, v0, a0, made


def avm_t1(net, thr, newlen=None, cap=16, allow_cap=False):
    """T1 passes on a copy of the network; returns (new network, transitions)."""
    net, t1, _ = avm_transitions(net, thr, newlen, 0.0, cap, allow_cap)
    return net, t1


def avm_step(net, theta, p0, v0, seed, step, A0=1.0, KA=1.0, KP=1.0, mu=1.0, Dr=1.0, dt=0.01, thr=0.04, newlen=None,
             cap=16, t2_area=0.0, counts=False):
    """One AVM step on copies: returns (network, theta, T1s), or with counts
    (network, theta, T1s, T2s).  p0, v0, A0: scalars or per cell."""
    net = net.copy()
    theta = np.array(theta, np.float64, copy=True)
    p0, v0, a0 = _cells(net, p0), _cells(net, v0), _cells(net, A0)
    newlen = 1.5 * thr if newlen is None else newlen
    par = np.array([KA, KP, mu, Dr, dt, thr, newlen, t2_area], np.float64)
    applied = np.zeros(2, np.int32)
    _check(lib().cgo_avm_step(net.n, net.V, net.Lx, net.Ly, _d(net.hx), _d(net.hy), _d(theta), _i(net.vc),
                              _i(net.vn), _i(net.cc), _i(net.cv), _d(p0), _d(v0), _d(a0), _d(par), int(seed),
                              int(step), int(cap), _i(applied)), "avm_step")
    if counts:
        return net, theta, int(applied[0]), int(applied[1])
    return net, theta, int(applied[0])
