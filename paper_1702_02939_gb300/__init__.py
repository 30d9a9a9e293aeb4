"""cellgb: GB300-native self-propelled Voronoi (SPV) model.

Thin Python binding of libcellgb.so (C ABI declared in include/cellgb.h).  The
functions ``cg_*`` below carry the same names and arguments as the C entry
points and only marshal pointers; all computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the CUDA stream.

Model: Sussman, "cellGPU: massively parallel simulations of dynamic vertex
models", arXiv 1702.02939 (energy Eq. 1, forces Eqs. A6-A16, motion Eq. 3,
topology test and repair Sec. 2.C.3-4).
"""
import ctypes as C
import os

import numpy as np

from . import _build

MAX_RING = 16
_LIB_PATH = _build.LIB
_lib = None

STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "ring overflow",
          -4: "repair cap exceeded", -5: "inconsistent rings", -6: "non-finite position",
          -7: "box too small", -8: "degenerate input", -9: "too many repair candidates",
          -10: "T1 candidates left after the pass cap"}


class CellgbError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"cellgb status {code} ({STATUS.get(code, '?')}) {msg}".strip())


class cg_replica(C.Structure):
    _fields_ = [("n", C.c_int32), ("Lx", C.c_double), ("Ly", C.c_double), ("p0", C.c_double),
                ("v0", C.c_double)]


class cg_params(C.Structure):
    _fields_ = [("A0", C.c_double), ("KA", C.c_double), ("KP", C.c_double), ("mu", C.c_double),
                ("Dr", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64),
                ("repair_cap", C.c_int32), ("sort_every", C.c_int32), ("precision", C.c_int32),
                ("reserved", C.c_int32)]


class cg_launch(C.Structure):
    _fields_ = [("repair_blocks_per_sm", C.c_int32), ("check_blocks_per_sm", C.c_int32),
                ("dir_blocks_per_sm", C.c_int32), ("dir_low_priority", C.c_int32),
                ("geom_blocks_per_sm", C.c_int32), ("test_blocks_per_sm", C.c_int32),
                ("dir_beside_geom", C.c_int32), ("ring_order", C.c_int32), ("force_beside", C.c_int32)]


class cg_avm_params(C.Structure):
    _fields_ = [("A0", C.c_double), ("KA", C.c_double), ("KP", C.c_double), ("mu", C.c_double),
                ("Dr", C.c_double), ("dt", C.c_double), ("t1_threshold", C.c_double),
                ("t1_length", C.c_double), ("seed", C.c_uint64), ("t1_cap", C.c_int32),
                ("cell_capacity", C.c_int32), ("t2_area", C.c_double), ("sort_every", C.c_int32)]


class cg_counters(C.Structure):
    _fields_ = [("steps", C.c_int64), ("flagged_total", C.c_int64), ("repaired_total", C.c_int64),
                ("last_flagged", C.c_int32), ("last_rounds", C.c_int32), ("status", C.c_int32),
                ("reserved", C.c_int32), ("loop_total", C.c_int64)]


def lib():
    """The loaded library.  Fails loudly if it was not built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libcellgb.so not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(_LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.cg_workspace_bytes.argtypes = [i32, C.POINTER(cg_replica), C.POINTER(C.c_size_t)]
        L.cg_create.argtypes = [i32, C.POINTER(cg_replica), C.POINTER(cg_params), vp, vp, vp, vp, C.c_size_t,
                                vp, C.POINTER(vp)]
        L.cg_step.argtypes = [vp, i64]
        L.cg_run_io.argtypes = [vp, i64, vp, i64, vp, vp, i64]
        L.cg_sync.argtypes = [vp]
        L.cg_profile_step.argtypes = [vp, i64, C.POINTER(C.c_double), i32]
        L.cg_get_state.argtypes = [vp, vp, vp, vp]
        L.cg_set_state.argtypes = [vp, vp, vp, vp]
        L.cg_get_geometry.argtypes = [vp, vp, vp]
        L.cg_get_forces.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        L.cg_get_neighbors.argtypes = [vp, vp, vp]
        L.cg_set_p0.argtypes = [vp, vp]
        L.cg_set_v0.argtypes = [vp, vp]
        L.cg_get_counters.argtypes = [vp, C.POINTER(cg_counters)]
        L.cg_director_terms.argtypes = [vp, i32, vp, vp, i64, vp, vp, vp]
        L.cg_backward_bytes.argtypes = [vp, i64, i32, C.POINTER(C.c_size_t)]
        L.cg_set_moduli.argtypes = [vp, C.c_double, C.c_double]
        L.cg_set_step.argtypes = [vp, i64]
        L.cg_run_checkpointed.argtypes = [vp, i64, i32, vp, C.c_size_t]
        L.cg_backward.argtypes = [vp, i64, i32, vp, C.c_size_t, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cg_hvp.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, C.c_size_t]
        for name in ("cg_backward_bytes", "cg_set_moduli", "cg_set_step", "cg_run_checkpointed", "cg_backward",
                     "cg_hvp"):
            getattr(L, name).restype = C.c_int
        L.cg_set_noise_ids.argtypes = [vp, vp]
        L.cg_set_frame.argtypes = [vp, i32, C.c_double, C.c_double, C.c_double, C.c_double]
        L.cg_halo_pack.argtypes = [vp, vp, vp]
        L.cg_halo_unpack.argtypes = [vp, vp, vp]
        for name in ("cg_set_noise_ids", "cg_set_frame", "cg_halo_pack", "cg_halo_unpack"):
            getattr(L, name).restype = C.c_int
        L.cg_triangulate_noalloc.argtypes = [i32, C.c_double, C.c_double, vp, vp, vp, vp, vp]
        L.cg_triangulate_noalloc.restype = C.c_int
        L.cg_num_cells.argtypes = [vp]
        L.cg_num_cells.restype = i64
        L.cg_destroy.argtypes = [vp]
        L.cg_status_string.argtypes = [C.c_int]
        L.cg_status_string.restype = C.c_char_p
        L.cg_last_error.argtypes = [vp]
        L.cg_last_error.restype = C.c_char_p
        for name in ("cg_workspace_bytes", "cg_create", "cg_step", "cg_sync", "cg_profile_step", "cg_get_state", "cg_set_state",
                     "cg_get_geometry", "cg_get_forces", "cg_get_neighbors", "cg_set_p0", "cg_set_v0",
                     "cg_get_counters", "cg_destroy"):
            getattr(L, name).restype = C.c_int
        L.cg_get_launch.argtypes = [vp, C.POINTER(cg_launch)]
        L.cg_set_launch.argtypes = [vp, C.POINTER(cg_launch)]
        L.cg_autotune_bytes.argtypes = [vp, C.c_size_t, C.POINTER(C.c_size_t)]
        L.cg_autotune.argtypes = [vp, i32, C.c_size_t, vp, C.c_size_t, C.POINTER(cg_launch), C.POINTER(C.c_double)]
        for name in ("cg_get_launch", "cg_set_launch", "cg_autotune_bytes", "cg_autotune"):
            getattr(L, name).restype = C.c_int
        # active vertex model
        L.cg_avm_workspace_bytes.argtypes = [i32, C.c_double, C.c_double, C.POINTER(C.c_size_t)]
        L.cg_avm_workspace_bytes_capacity.argtypes = [i32, i32, C.c_double, C.c_double, C.POINTER(C.c_size_t)]
        L.cg_avm_create.argtypes = [i32, C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(cg_avm_params),
                                    vp, vp, vp, vp, C.c_size_t, vp, C.POINTER(vp)]
        L.cg_avm_step.argtypes = [vp, i64]
        L.cg_avm_sync.argtypes = [vp]
        L.cg_avm_profile_step.argtypes = [vp, i64, C.POINTER(C.c_double), i32]
        L.cg_avm_get_state.argtypes = [vp, vp, vp, vp]
        L.cg_avm_get_topology.argtypes = [vp, vp, vp, vp, vp]
        L.cg_avm_set_state.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.cg_avm_get_geometry.argtypes = [vp, vp, vp]
        L.cg_avm_get_forces.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
        L.cg_avm_t1.argtypes = [vp]
        L.cg_avm_set_p0.argtypes = [vp, vp]
        L.cg_avm_set_v0.argtypes = [vp, vp]
        L.cg_avm_set_a0.argtypes = [vp, vp]
        L.cg_avm_set_step.argtypes = [vp, i64]
        L.cg_avm_get_cell_params.argtypes = [vp, vp, vp, vp]
        L.cg_avm_divide.argtypes = [vp, i32, vp, vp, vp, C.POINTER(i32)]
        L.cg_avm_get_counters.argtypes = [vp, C.POINTER(cg_counters)]
        L.cg_avm_sort.argtypes = [vp]
        L.cg_avm_get_tags.argtypes = [vp, vp, vp]
        L.cg_avm_destroy.argtypes = [vp]
        L.cg_avm_last_error.argtypes = [vp]
        L.cg_avm_last_error.restype = C.c_char_p
        for name in ("cg_avm_workspace_bytes", "cg_avm_workspace_bytes_capacity", "cg_avm_create", "cg_avm_step", "cg_avm_sync", "cg_avm_get_state",
                     "cg_avm_get_topology", "cg_avm_set_state", "cg_avm_get_geometry", "cg_avm_get_forces",
                     "cg_avm_t1", "cg_avm_set_p0", "cg_avm_set_v0", "cg_avm_set_a0", "cg_avm_divide", "cg_avm_set_step", "cg_avm_get_cell_params", "cg_avm_get_counters", "cg_avm_destroy",
                     "cg_avm_profile_step"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# C-named wrappers (argument marshalling only)
# ---------------------------------------------------------------------------
def _ptr(a):
    """Raw address of a torch tensor or numpy array (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


def _check(rc, ctx=None):
    if rc != 0:
        msg = lib().cg_last_error(ctx).decode() if ctx else ""
        raise CellgbError(rc, msg)


def _reps(replicas):
    arr = (cg_replica * len(replicas))()
    for k, r in enumerate(replicas):
        arr[k] = cg_replica(int(r["n"]), float(r["Lx"]), float(r["Ly"]), float(r["p0"]), float(r["v0"]))
    return arr


def cg_workspace_bytes(replicas):
    out = C.c_size_t(0)
    _check(lib().cg_workspace_bytes(len(replicas), _reps(replicas), C.byref(out)))
    return out.value


def cg_create(replicas, params, x, y, theta, workspace, stream):
    ctx = C.c_void_p()
    _check(lib().cg_create(len(replicas), _reps(replicas), C.byref(params), _ptr(x), _ptr(y), _ptr(theta),
                           _ptr(workspace), workspace.numel(), C.c_void_p(stream), C.byref(ctx)))
    return ctx


def cg_step(ctx, nsteps):
    _check(lib().cg_step(ctx, int(nsteps)), ctx)


PHASES = ("geometry", "force_move", "test", "cell_list", "repair", "directors", "ring_order")


def cg_profile_step(ctx, nsteps):
    ms = (C.c_double * len(PHASES))()
    _check(lib().cg_profile_step(ctx, int(nsteps), ms, len(PHASES)), ctx)
    return {k: ms[i] for i, k in enumerate(PHASES)}


def cg_sync(ctx):
    _check(lib().cg_sync(ctx), ctx)


def cg_get_state(ctx, x, y, theta):
    _check(lib().cg_get_state(ctx, _ptr(x), _ptr(y), _ptr(theta)), ctx)


def cg_set_state(ctx, x, y, theta):
    _check(lib().cg_set_state(ctx, _ptr(x), _ptr(y), _ptr(theta)), ctx)


def cg_get_geometry(ctx, A, P):
    _check(lib().cg_get_geometry(ctx, _ptr(A), _ptr(P)), ctx)


def cg_get_forces(ctx, Fx, Fy):
    e = C.c_double(0.0)
    _check(lib().cg_get_forces(ctx, _ptr(Fx), _ptr(Fy), C.byref(e)), ctx)
    return e.value


def cg_get_neighbors(ctx, cnt, nbr):
    _check(lib().cg_get_neighbors(ctx, _ptr(cnt), _ptr(nbr)), ctx)


def cg_set_p0(ctx, p0):
    _check(lib().cg_set_p0(ctx, _ptr(p0)), ctx)


def cg_set_v0(ctx, v0):
    _check(lib().cg_set_v0(ctx, _ptr(v0)), ctx)


def cg_get_counters(ctx):
    c = cg_counters()
    _check(lib().cg_get_counters(ctx, C.byref(c)), ctx)
    return {k: getattr(c, k) for k, _ in cg_counters._fields_ if k != "reserved"}


def cg_run_io(ctx, nsteps, v0, v0_stride, x, y, out_stride):
    _check(lib().cg_run_io(ctx, int(nsteps), _ptr(v0), int(v0_stride), _ptr(x), _ptr(y), int(out_stride)), ctx)


def cg_director_terms(ctx, n, theta, tag, step, cs, sn, xi):
    _check(lib().cg_director_terms(ctx, int(n), _ptr(theta), _ptr(tag), int(step), _ptr(cs), _ptr(sn), _ptr(xi)),
           ctx)


def cg_backward_bytes(ctx, nsteps, ckpt_every):
    out = C.c_size_t(0)
    _check(lib().cg_backward_bytes(ctx, int(nsteps), int(ckpt_every), C.byref(out)), ctx)
    return out.value


def cg_set_moduli(ctx, KA, KP):
    _check(lib().cg_set_moduli(ctx, float(KA), float(KP)), ctx)


def cg_set_step(ctx, step):
    _check(lib().cg_set_step(ctx, int(step)), ctx)


def cg_set_noise_ids(ctx, ids):
    _check(lib().cg_set_noise_ids(ctx, _ptr(ids)), ctx)


def cg_set_frame(ctx, replica, x0, y0, Lx_outer, Ly_outer):
    _check(lib().cg_set_frame(ctx, int(replica), float(x0), float(y0), float(Lx_outer), float(Ly_outer)), ctx)


def cg_halo_pack(ctx, slot, out):
    _check(lib().cg_halo_pack(ctx, _ptr(slot), _ptr(out)), ctx)


def cg_halo_unpack(ctx, slot, inp):
    _check(lib().cg_halo_unpack(ctx, _ptr(slot), _ptr(inp)), ctx)


def cg_run_checkpointed(ctx, nsteps, ckpt_every, bw):
    _check(lib().cg_run_checkpointed(ctx, int(nsteps), int(ckpt_every), _ptr(bw), bw.numel()), ctx)


def cg_backward(ctx, nsteps, ckpt_every, bw, gxT, gyT, gAT, gPT, gx0, gy0, gp0, gv0):
    gK = (C.c_double * 2)()
    _check(lib().cg_backward(ctx, int(nsteps), int(ckpt_every), _ptr(bw), bw.numel(), _ptr(gxT), _ptr(gyT),
                             _ptr(gAT), _ptr(gPT), _ptr(gx0), _ptr(gy0), _ptr(gp0), _ptr(gv0), gK), ctx)
    return float(gK[0]), float(gK[1])


def cg_hvp(ctx, vx, vy, hvx, hvy, Adot, Pdot, bw):
    _check(lib().cg_hvp(ctx, _ptr(vx), _ptr(vy), _ptr(hvx), _ptr(hvy), _ptr(Adot), _ptr(Pdot), _ptr(bw),
                        bw.numel()), ctx)


NOALLOC_MAX_CELLS = 16384


def cg_triangulate_noalloc(n, Lx, Ly, x, y, cnt, nbr, stream):
    """Delaunay rings of n cells without any device allocation (scratch is a
    static array of the library, shared by all calls; at most
    NOALLOC_MAX_CELLS cells).  x, y, cnt, nbr are device tensors."""
    if n > NOALLOC_MAX_CELLS:
        raise CellgbError(-1, f"n={n} exceeds the static scratch limit of {NOALLOC_MAX_CELLS} cells")
    _check(lib().cg_triangulate_noalloc(int(n), float(Lx), float(Ly), _ptr(x), _ptr(y), _ptr(cnt), _ptr(nbr),
                                        C.c_void_p(stream)))


def cg_get_launch(ctx):
    out = cg_launch()
    _check(lib().cg_get_launch(ctx, C.byref(out)), ctx)
    return {k: getattr(out, k) for k, _ in cg_launch._fields_}


def cg_set_launch(ctx, launch):
    _check(lib().cg_set_launch(ctx, C.byref(cg_launch(**launch))), ctx)


def cg_autotune_bytes(ctx, flush_bytes=0):
    out = C.c_size_t(0)
    _check(lib().cg_autotune_bytes(ctx, int(flush_bytes), C.byref(out)), ctx)
    return out.value


def cg_autotune(ctx, steps_per_trial, flush_bytes, scratch):
    best, ms = cg_launch(), C.c_double(0.0)
    _check(lib().cg_autotune(ctx, int(steps_per_trial), int(flush_bytes), _ptr(scratch), scratch.numel(),
                             C.byref(best), C.byref(ms)), ctx)
    return {k: getattr(best, k) for k, _ in cg_launch._fields_}, ms.value


def cg_num_cells(ctx):
    return int(lib().cg_num_cells(ctx))


def cg_destroy(ctx):
    if ctx:
        lib().cg_destroy(ctx)


# ---------------------------------------------------------------------------
# Convenience object
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Persisted launch shapes: the autotuner's choice per GPU model and problem
# class, so that a run can reuse a tuning instead of repeating it.
# ---------------------------------------------------------------------------
LAUNCH_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "launch_cache.json")


def launch_cache_key(gpu_name, n, replicas, precision, flush_bytes):
    """GPU model | precision | replica count bucket | cell count bucket (the
    nearest power of two) | whether the L2 is evicted before each step."""
    import math

    name = str(gpu_name).replace("|", "/")
    rb = 1 if replicas <= 1 else 2 ** int(round(math.log2(replicas)))
    nb = 2 ** int(round(math.log2(max(int(n), 1))))
    return f"{name}|{'f32' if precision == 1 else 'f64'}|R~{rb}|N~{nb}|l2{'cold' if flush_bytes else 'warm'}"


def _read_launch_cache(path):
    import json

    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _write_launch_cache(path, key, launch):
    import json

    data = _read_launch_cache(path)
    data[key] = {k: int(v) for k, v in launch.items()}
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class SPV:
    """One or more independent periodic SPV systems advanced together.

    replicas: list of dicts {n, Lx, Ly, p0, v0}; x, y, theta: arrays of the
    concatenated cells (numpy, or torch tensors on any device).
    """

    def __init__(self, replicas, x, y, theta, A0=1.0, KA=1.0, KP=1.0, mu=1.0, Dr=1.0, dt=0.01, seed=0,
                 repair_cap=4, sort_every=0, precision="f64", device="cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.replicas = [dict(r) for r in replicas]
        if precision not in ("f64", "f32"):
            raise ValueError("precision is 'f64' or 'f32'")
        self.params = cg_params(A0, KA, KP, mu, Dr, dt, int(seed), int(repair_cap), int(sort_every),
                                1 if precision == "f32" else 0, 0)
        nbytes = cg_workspace_bytes(self.replicas)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.n = sum(int(r["n"]) for r in self.replicas)
        self.stream = torch.cuda.current_stream(self.device).cuda_stream
        xs, ys, ts = (self._as_input(v) for v in (x, y, theta))
        self.ctx = cg_create(self.replicas, self.params, xs, ys, ts, self.workspace, self.stream)

    def _as_input(self, v):
        t = self.torch
        if isinstance(v, t.Tensor):
            return v.to(dtype=t.float64).contiguous()
        return np.ascontiguousarray(v, dtype=np.float64)

    def _out(self, n=None, dtype=None):
        t = self.torch
        return t.empty(self.n if n is None else n, dtype=dtype or t.float64, device=self.device)

    def step(self, nsteps=1):
        cg_step(self.ctx, nsteps)

    def sync(self):
        cg_sync(self.ctx)

    def profile(self, nsteps):
        return cg_profile_step(self.ctx, nsteps)

    def run_io(self, nsteps, v0=None, x=None, y=None, v0_stride=0, out_stride=0):
        """nsteps steps with per-step I/O overlapped with the kernels: v0 of
        step k from v0[k * v0_stride:], positions after step k into
        x[k * out_stride:], y[k * out_stride:] (contiguous float64 tensors or
        arrays, host memory page-locked for overlap, or None)."""
        cg_run_io(self.ctx, nsteps, v0, v0_stride, x, y, out_stride)

    def state(self):
        x, y, th = self._out(), self._out(), self._out()
        cg_get_state(self.ctx, x, y, th)
        return x, y, th

    def set_state(self, x, y, theta=None):
        cg_set_state(self.ctx, self._as_input(x), self._as_input(y),
                     None if theta is None else self._as_input(theta))

    def geometry(self):
        A, P = self._out(), self._out()
        cg_get_geometry(self.ctx, A, P)
        return A, P

    def forces(self):
        Fx, Fy = self._out(), self._out()
        E = cg_get_forces(self.ctx, Fx, Fy)
        return Fx, Fy, E

    def neighbors(self):
        t = self.torch
        cnt = self._out(dtype=t.int32)
        nbr = self._out(self.n * MAX_RING, dtype=t.int32)
        cg_get_neighbors(self.ctx, cnt, nbr)
        return cnt, nbr.view(self.n, MAX_RING)

    def set_p0(self, p0):
        cg_set_p0(self.ctx, self._as_input(p0))

    def set_v0(self, v0):
        cg_set_v0(self.ctx, self._as_input(v0))

    def counters(self):
        return cg_get_counters(self.ctx)

    def director_terms(self, theta, tag, step):
        """(cos theta, sin theta, xi(seed, tag, step)) as the FP64 step
        evaluates them, for device tensors theta (float64) and tag (int32)."""
        t = self.torch
        theta = theta.to(device=self.device, dtype=t.float64).contiguous()
        tag = tag.to(device=self.device, dtype=t.int32).contiguous()
        n = theta.numel()
        if tag.numel() != n:
            raise ValueError("theta and tag differ in length")
        cs, sn, xi = self._out(n), self._out(n), self._out(n)
        cg_director_terms(self.ctx, n, theta, tag, step, cs, sn, xi)
        self.sync()
        return cs, sn, xi

    @property
    def launch(self):
        return cg_get_launch(self.ctx)

    def set_launch(self, **launch):
        cur = cg_get_launch(self.ctx)
        cur.update(launch)
        cg_set_launch(self.ctx, cur)

    def autotune(self, steps_per_trial=10, flush_bytes=0, cache=None):
        """Times candidate launch shapes on a temporary copy of the current
        state and keeps the fastest; the simulation itself takes no step.
        flush_bytes > 0 times every step after an L2-evicting write.

        cache: path of a JSON file of tuned shapes (see `launch_cache_key`).
        A stored entry for this GPU and problem class is applied without
        timing (ms is then None); otherwise the tuned shapes are stored.
        Launch shapes change timing only, never results."""
        key = None
        if cache is not None:
            key = launch_cache_key(self.torch.cuda.get_device_name(self.device), self.n, len(self.replicas),
                                   self.params.precision, flush_bytes)
            hit = _read_launch_cache(cache).get(key)
            if hit is not None:
                known = {f for f, _ in cg_launch._fields_}
                self.set_launch(**{k: v for k, v in hit.items() if k in known})
                return self.launch, None
        t = self.torch
        scratch = t.empty(cg_autotune_bytes(self.ctx, flush_bytes), dtype=t.uint8, device=self.device)
        best, ms = cg_autotune(self.ctx, steps_per_trial, flush_bytes, scratch)
        del scratch
        if key is not None:
            _write_launch_cache(cache, key, best)
        return best, ms

    def set_moduli(self, KA, KP):
        cg_set_moduli(self.ctx, KA, KP)

    def set_step(self, step):
        cg_set_step(self.ctx, step)

    def set_noise_ids(self, ids):
        """Philox counters of the cells' director noise (user order), in place
        of their user indices."""
        t = self.torch
        ids = t.as_tensor(ids, dtype=t.int32).contiguous()
        cg_set_noise_ids(self.ctx, ids)

    def set_frame(self, x0, y0, Lx_outer, Ly_outer, replica=0):
        """Makes the replica's box the frame at (x0, y0) of a larger periodic
        box: moves are rounded in the larger box's coordinates."""
        cg_set_frame(self.ctx, replica, x0, y0, Lx_outer, Ly_outer)

    def halo_pack(self, slot, out):
        """Pending positions (int64 grid coordinates of the larger box) of the
        cells with slot[u] >= 0 into out[2 slot:2 slot + 2] (device tensors;
        asynchronous on the context's stream)."""
        cg_halo_pack(self.ctx, slot, out)

    def halo_unpack(self, slot, inp):
        """Replaces the pending positions of the cells with slot[u] >= 0 by
        inp[2 slot:2 slot + 2] (device tensors; asynchronous)."""
        cg_halo_unpack(self.ctx, slot, inp)

    def _bwd_buffer(self, nsteps, ckpt_every):
        nbytes = cg_backward_bytes(self.ctx, nsteps, ckpt_every)
        return self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)

    def hvp(self, vx, vy):
        """(H v, dA/dv, dP/dv) at the current state."""
        bw = self._bwd_buffer(1, 1)
        out = [self._out() for _ in range(4)]
        cg_hvp(self.ctx, self._as_input(vx), self._as_input(vy), *out, bw)
        return tuple(out)

    def run_checkpointed(self, nsteps, ckpt_every):
        bw = self._bwd_buffer(nsteps, ckpt_every)
        cg_run_checkpointed(self.ctx, nsteps, ckpt_every, bw)
        return bw

    def backward(self, bw, nsteps, ckpt_every, gxT, gyT, gAT, gPT):
        """Cotangents (gx0, gy0, gp0, gv0, gKA, gKP) of a checkpointed run."""
        out = [self._out() for _ in range(4)]
        gKA, gKP = cg_backward(self.ctx, nsteps, ckpt_every, bw, *(self._as_input(g) for g in (gxT, gyT, gAT, gPT)),
                               *out)
        return (*out, gKA, gKP)

    def close(self):
        if getattr(self, "ctx", None):
            cg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class SPVRunFunction(torch.autograd.Function):
        """Differentiable SPV run: (x0, y0, p0, v0, KA, KP) -> (x, y, A, P) after
        nsteps steps of Eq. 3 with the director noise fixed by the seed.  The
        backward is the library's checkpointed reverse pass (H g products on
        the frozen topology of each step), exact on windows without neighbour
        changes.  p0 is per cell; v0, KA, KP are scalars (tensors)."""

        @staticmethod
        def forward(fctx, x0, y0, p0, v0, KA, KP, sim, theta0, nsteps, ckpt_every, step0):
            n = sim.n
            sim.set_moduli(float(KA), float(KP))
            sim.set_p0(p0.detach())
            sim.set_v0(torch.full((n,), float(v0), dtype=torch.float64, device=sim.device))
            sim.set_state(x0.detach(), y0.detach(), theta0)
            sim.set_step(step0)
            bw = sim.run_checkpointed(nsteps, ckpt_every)
            x, y, _ = sim.state()
            A, P = sim.geometry()
            fctx.sim, fctx.bw, fctx.nsteps, fctx.every = sim, bw, nsteps, ckpt_every
            return x, y, A, P

        @staticmethod
        def backward(fctx, gx, gy, gA, gP):
            sim = fctx.sim
            z = lambda g: torch.zeros(sim.n, dtype=torch.float64, device=sim.device) if g is None else g.contiguous()
            gx0, gy0, gp0, gv0, gKA, gKP = sim.backward(fctx.bw, fctx.nsteps, fctx.every, z(gx), z(gy), z(gA), z(gP))
            t = lambda v: torch.tensor(v, dtype=torch.float64)
            return gx0, gy0, gp0, gv0.sum().cpu(), t(gKA), t(gKP), None, None, None, None, None

    return SPVRunFunction


def spv_run_differentiable(sim, x0, y0, p0, v0, KA, KP, theta0, nsteps, ckpt_every=50, step0=0):
    """Differentiable nsteps-step SPV run; returns final (x, y, A, P)."""
    return _autograd_function().apply(x0, y0, p0, v0, KA, KP, sim, theta0, nsteps, ckpt_every, step0)


# ---------------------------------------------------------------------------
# Active vertex model (Sec. 2.D, Eq. 4, Fig. 1): C-named wrappers
# ---------------------------------------------------------------------------
def _check_avm(rc, ctx=None):
    if rc != 0:
        msg = lib().cg_avm_last_error(ctx).decode() if ctx else ""
        raise CellgbError(rc, msg)


def cg_avm_workspace_bytes(n, Lx, Ly):
    out = C.c_size_t(0)
    _check_avm(lib().cg_avm_workspace_bytes(int(n), float(Lx), float(Ly), C.byref(out)))
    return out.value


def cg_avm_workspace_bytes_capacity(n, capacity, Lx, Ly):
    out = C.c_size_t(0)
    _check_avm(lib().cg_avm_workspace_bytes_capacity(int(n), int(capacity), float(Lx), float(Ly), C.byref(out)))
    return out.value


def cg_avm_create(n, Lx, Ly, p0, v0, params, x, y, theta, workspace, stream):
    ctx = C.c_void_p()
    _check_avm(lib().cg_avm_create(int(n), float(Lx), float(Ly), float(p0), float(v0), C.byref(params), _ptr(x),
                                   _ptr(y), _ptr(theta), _ptr(workspace), workspace.numel(), C.c_void_p(stream),
                                   C.byref(ctx)))
    return ctx


def cg_avm_step(ctx, nsteps):
    _check_avm(lib().cg_avm_step(ctx, int(nsteps)), ctx)


def cg_avm_profile_step(ctx, nsteps):
    out = (C.c_double * 5)()
    _check_avm(lib().cg_avm_profile_step(ctx, int(nsteps), out, 5), ctx)
    return {"cells_ms": out[0], "vertices_ms": out[1], "t1_ms": out[2], "t1_passes": out[3], "dir_ms": out[4]}


def cg_avm_sync(ctx):
    _check_avm(lib().cg_avm_sync(ctx), ctx)


def cg_avm_get_state(ctx, hx, hy, theta):
    _check_avm(lib().cg_avm_get_state(ctx, _ptr(hx), _ptr(hy), _ptr(theta)), ctx)


def cg_avm_get_topology(ctx, vc, vn, cc, cv):
    _check_avm(lib().cg_avm_get_topology(ctx, _ptr(vc), _ptr(vn), _ptr(cc), _ptr(cv)), ctx)


def cg_avm_set_state(ctx, hx, hy, theta, vc, vn, cc, cv):
    _check_avm(lib().cg_avm_set_state(ctx, _ptr(hx), _ptr(hy), _ptr(theta), _ptr(vc), _ptr(vn), _ptr(cc),
                                      _ptr(cv)), ctx)


def cg_avm_get_geometry(ctx, A, P):
    _check_avm(lib().cg_avm_get_geometry(ctx, _ptr(A), _ptr(P)), ctx)


def cg_avm_get_forces(ctx, Fx, Fy):
    E = C.c_double(0.0)
    _check_avm(lib().cg_avm_get_forces(ctx, _ptr(Fx), _ptr(Fy), C.byref(E)), ctx)
    return E.value


def cg_avm_t1(ctx):
    _check_avm(lib().cg_avm_t1(ctx), ctx)


def cg_avm_set_p0(ctx, p0):
    _check_avm(lib().cg_avm_set_p0(ctx, _ptr(p0)), ctx)


def cg_avm_set_v0(ctx, v0):
    _check_avm(lib().cg_avm_set_v0(ctx, _ptr(v0)), ctx)


def cg_avm_set_a0(ctx, a0):
    _check_avm(lib().cg_avm_set_a0(ctx, _ptr(a0)), ctx)


def cg_avm_set_step(ctx, step):
    _check_avm(lib().cg_avm_set_step(ctx, int(step)), ctx)


def cg_avm_get_cell_params(ctx, p0, v0, a0):
    _check_avm(lib().cg_avm_get_cell_params(ctx, _ptr(p0), _ptr(v0), _ptr(a0)), ctx)


def cg_avm_divide(ctx, count, cells, dirs, made):
    n_made = C.c_int32(0)
    _check_avm(lib().cg_avm_divide(ctx, int(count), _ptr(cells), _ptr(dirs), _ptr(made), C.byref(n_made)), ctx)
    return n_made.value


def cg_avm_get_counters(ctx):
    c = cg_counters()
    _check_avm(lib().cg_avm_get_counters(ctx, C.byref(c)), ctx)
    return {"steps": c.steps, "t1_total": c.repaired_total, "t2_total": c.flagged_total, "t1_passes": c.last_rounds,
            "status": c.status, "loop_total": c.loop_total}


def cg_avm_sort(ctx):
    _check_avm(lib().cg_avm_sort(ctx), ctx)


def cg_avm_get_tags(ctx, vtag, ctag):
    _check_avm(lib().cg_avm_get_tags(ctx, _ptr(vtag), _ptr(ctag)), ctx)


def cg_avm_destroy(ctx):
    if ctx:
        lib().cg_avm_destroy(ctx)


class AVM:
    """A periodic active vertex model started from the Voronoi tessellation of
    seed positions x, y (numpy, or torch tensors on any device)."""

    def __init__(self, n, Lx, Ly, x, y, theta, p0=3.8, v0=0.1, A0=1.0, KA=1.0, KP=1.0, mu=1.0, Dr=1.0, dt=0.01,
                 t1_threshold=0.04, t1_length=0.0, seed=0, t1_cap=16, t2_area=0.0, capacity=None, sort_every=0,
                 device="cuda"):
        """n seeds; `capacity` cell slots (default n) leave room for divisions:
        per-cell outputs then have `capacity` entries, per-vertex ones 2x.
        sort_every > 0: Hilbert re-sort of the storage at creation and every
        sort_every steps (results unchanged; ids stay those of the API)."""
        import torch
        self.torch = torch
        self.device = torch.device(device)
        cap = int(n) if capacity is None else int(capacity)
        self.n_seed = int(n)
        self.n, self.V = cap, 2 * cap
        self.params = cg_avm_params(A0, KA, KP, mu, Dr, dt, t1_threshold, t1_length, int(seed), int(t1_cap), cap,
                                    float(t2_area), int(sort_every))
        nbytes = cg_avm_workspace_bytes_capacity(n, cap, Lx, Ly)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device).cuda_stream
        xs, ys, ts = (self._as_input(v) for v in (x, y, theta))
        self.ctx = cg_avm_create(n, Lx, Ly, p0, v0, self.params, xs, ys, ts, self.workspace, self.stream)

    def _as_input(self, v, dtype=None):
        t = self.torch
        if isinstance(v, t.Tensor):
            return v.to(dtype=dtype or t.float64).contiguous()
        return np.ascontiguousarray(v, dtype=np.int32 if dtype is t.int32 else np.float64)

    def _out(self, n, dtype=None):
        t = self.torch
        return t.empty(n, dtype=dtype or t.float64, device=self.device)

    def step(self, nsteps=1):
        cg_avm_step(self.ctx, nsteps)

    def sync(self):
        cg_avm_sync(self.ctx)

    def profile(self, nsteps):
        return cg_avm_profile_step(self.ctx, nsteps)

    def state(self):
        hx, hy, th = self._out(self.V), self._out(self.V), self._out(self.n)
        cg_avm_get_state(self.ctx, hx, hy, th)
        return hx, hy, th

    def sort(self):
        """Hilbert re-sort of the storage now (ids and results unchanged)."""
        cg_avm_sort(self.ctx)

    def storage_tags(self):
        """(vertex tags [V], cell tags [N]) by storage slot (int32 tensors)."""
        t = self.torch
        vt, ct = self._out(self.V, t.int32), self._out(self.n, t.int32)
        cg_avm_get_tags(self.ctx, vt, ct)
        return vt, ct

    def topology(self):
        """(vc [V,3], vn [V,3], cc [N], cv [N, MAX_RING]) as int32 tensors."""
        t = self.torch
        vc, vn = self._out(3 * self.V, t.int32), self._out(3 * self.V, t.int32)
        cc, cv = self._out(self.n, t.int32), self._out(self.n * MAX_RING, t.int32)
        cg_avm_get_topology(self.ctx, vc, vn, cc, cv)
        return vc.view(self.V, 3), vn.view(self.V, 3), cc, cv.view(self.n, MAX_RING)

    def set_state(self, hx, hy, theta=None, vc=None, vn=None, cc=None, cv=None):
        t = self.torch
        ints = [None if a is None else self._as_input(a, t.int32) for a in (vc, vn, cc, cv)]
        cg_avm_set_state(self.ctx, self._as_input(hx), self._as_input(hy),
                         None if theta is None else self._as_input(theta), *ints)

    def geometry(self):
        A, P = self._out(self.n), self._out(self.n)
        cg_avm_get_geometry(self.ctx, A, P)
        return A, P

    def forces(self):
        Fx, Fy = self._out(self.V), self._out(self.V)
        E = cg_avm_get_forces(self.ctx, Fx, Fy)
        return Fx, Fy, E

    def t1(self):
        cg_avm_t1(self.ctx)

    def set_p0(self, p0):
        cg_avm_set_p0(self.ctx, self._as_input(p0))

    def set_v0(self, v0):
        cg_avm_set_v0(self.ctx, self._as_input(v0))

    def divide(self, cells, dirs):
        """Divides cells[k] along dirs[k] = (ux, uy), in order; returns the
        int32 array made[k] (1 when division k was made).  The new cells take
        the next free slots (see `capacity`)."""
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1)
        if dirs.size != 2 * cells.size:
            raise ValueError("one direction (ux, uy) per cell")
        made = np.zeros(cells.size, np.int32)
        cg_avm_divide(self.ctx, cells.size, cells, dirs, made)
        return made

    def cell_params(self):
        """(p0, v0, A0) per cell slot as they stand (divisions copy them)."""
        p0, v0, a0 = self._out(self.n), self._out(self.n), self._out(self.n)
        cg_avm_get_cell_params(self.ctx, p0, v0, a0)
        return p0, v0, a0

    def set_step(self, step):
        """Sets the step counter that keys the director noise (to resume a run)."""
        cg_avm_set_step(self.ctx, step)

    def set_a0(self, a0):
        """Per-cell preferred areas (a cell given a small A0 shrinks and,
        with t2_area > 0, is removed once it is a small triangle)."""
        cg_avm_set_a0(self.ctx, self._as_input(a0))

    def counters(self):
        return cg_avm_get_counters(self.ctx)

    def close(self):
        if self.ctx:
            self.torch.cuda.synchronize(self.device)
            cg_avm_destroy(self.ctx)
            self.ctx = None
