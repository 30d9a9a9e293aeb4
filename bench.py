#!/usr/bin/env python3
"""SPV benchmark: cell-steps/s of the self-propelled Voronoi step on GB300.

Workload (Sussman, arXiv 1702.02939, SPV model of Sec. 2.C, fluid regime of
Fig. 3): N = 262144 cells at unit density in a periodic box L = 512, uniform
random positions and directors, p0 = 3.85, v0 = 0.1, A0 = K_A = K_P = mu =
D_r = 1, dt = 0.01, FP64.  The workload's 100 equilibration steps always run
first (--warmup adds untimed steps on top); every timed step runs the whole
hot path (geometry, force sets, net force, move, exact circumcircle test,
local repair) and is timed alone with CUDA events, with L2 flushed in
between.  The end-to-end figure replays the same timed steps from the same
state through the public API with host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain restatement of the method used
by the tests) on bounded spatial-window samples of the same workload.
With N > 1 (torchrun), each rank advances its own independent replica
(replicas only, weak scaling); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_CELLS = 262144
P0, V0, DT = 3.85, 0.1, 0.01
METRIC = "SPV cell-steps/s at N=262144 (FP64, 1 GB300)"
UNIT = "cell-steps/s"
WORKLOAD = "spv_fluid_N262144_L512_p0_3.85_v0_0.1_dt0.01_fp64"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FLUSH_BYTES = 256 * 1024 * 1024  # written between timed steps: more than the 126 MB L2
# The workload runs 100 equilibration steps before its timed steps, whatever
# the number of warm-up steps asked for.
EQUIL_STEPS = 100

# Algorithmic FP64 floating-point operations per cell-step of each kernel
# (fma = 2, add/mul/div/sqrt/rsqrt = 1, transcendental = 1), for the mean ring
# size of 6 of a random Voronoi tessellation.  Geometry counts each Delaunay
# circumcentre once (2 triangles per cell x 24, plus 6 ring slots x 36 for
# the Jacobian factors, area, edges and force sets, plus 13 per cell), not
# the three times the kernel evaluates it.
FLOPS_PER_CELL = {"geometry": 277.0, "force_move": 93.0}
# AVM: per cell of k_avm_cells (12 per polygon vertex x 6: offsets, shoelace
# term, edge, sqrt, sum; 12 for A, P and the coefficients) and per vertex of
# k_avm_force_move (3 edges x (offset, length, rsqrt, unit vector) + 3 force
# terms x 8 + activity and move).
AVM_FLOPS = {"cells_per_cell": 84.0, "vertices_per_vertex": 62.0}
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the AVM kernels at N = 65536 from one ncu capture of the current kernels
# (caches flushed before the kernel); None whenever a kernel has changed.
AVM_DRAM_BYTES_PER_LAUNCH = {"k_avm_cells": 8.14e6, "k_avm_force_move": 7.37e6}
# AVM storage order: Hilbert re-sort of the vertex and cell slots at creation
# and every this many steps (Sec. 2.B; results are the same either way).
AVM_SORT_EVERY = 100
# Algorithmic bytes per cell-step of the whole step (state read + written once).
BYTES_PER_CELL_STEP = 84.0
# FP64 peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Dominant-kernel DRAM traffic per launch (dram__bytes_read.sum +
# dram__bytes_write.sum) from one ncu capture of the current k_geom at
# N = 262144; None whenever the kernel has changed since the capture.
GEOM_DRAM_BYTES_PER_LAUNCH = 43.99e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS)
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=2000, help="length of the batched run")
    ap.add_argument("--batched-window", type=int, default=10, help="steps of the per-replica loop timed")
    ap.add_argument("--bwd-steps", type=int, default=1000)
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--no-avm", action="store_true")
    ap.add_argument("--domains", type=int, default=2, help="strip domains of the decomposed-run section (0: skip)")
    ap.add_argument("--domain-steps", type=int, default=200)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=500)
    ap.add_argument("--avm-steps", type=int, default=4900,
                    help="timed AVM steps after --avm-warmup (default: a 5000-step run)")
    ap.add_argument("--avm-warmup", type=int, default=100)
    ap.add_argument("--avm-profile-steps", type=int, default=20)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--retune", action="store_true",
                    help="tune the launch shapes afresh instead of taking the stored ones")
    ap.add_argument("--eager", action="store_true",
                    help="launch every kernel of the step eagerly instead of replaying the step graph "
                         "(same kernels and results; for kernel-level profilers)")
    ap.add_argument("--sweep", action="store_true",
                    help="time per step against N (solid and fluid regimes) and against p0, GPU and CPU "
                         "oracle; prints one JSON object (a study, not the bench line)")
    ap.add_argument("--avm-only", action="store_true",
                    help="run only the AVM section and print its JSON object (a diagnostic, not the bench line)")
    return ap.parse_args()


def launch_cache(args):
    """The persisted launch shapes (tuned per GPU model and problem class)
    unless --retune asks for a fresh tuning pass (which does not write)."""
    if args.retune:
        return None
    import paper_1702_02939_gb300 as cg

    return cg.LAUNCH_CACHE


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world, device):
    """The largest value over all ranks (timed regions are reported as the
    slowest rank's); one rank returns its own value."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, cells_per_rank, steps, ms):
    """Whole-job throughput: every rank advances its own system of
    cells_per_rank cells for `steps` steps in `ms` milliseconds (max over ranks)."""
    return world * cells_per_rank * steps / (ms * 1e-3)


def hbm_peak():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(n, seed):
    import workloads

    x, y, th, L = workloads.spv_uniform(n, seed)
    return x, y, th, L


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [t.strip() for t in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def kernels_launched(steps, loop_iterations, eager=False, ring_order=1, force_beside=0):
    # per step: begin-topology, test, 4 cell-list kernels, directors, the
    # ring-size grouping (if on), geometry of the new state, force + move;
    # graph only: the geometry fix-up of rewritten rings and, with the force
    # pass beside the rounds, the fix-up list and the force fix-up; per
    # repair round: repair + check
    graph_extra = 0 if eager else 1 + (2 if force_beside else 0)
    return (9 + (1 if ring_order else 0) + graph_extra) * steps + 2 * loop_iterations


def host_cpu():
    """Logical CPUs and model of the host the oracle runs on."""
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "processor name"):
                    model = f"{platform.machine()} {line.split(':', 1)[1].strip()}"
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def cpu_baseline(x, y, th, L, seconds):
    """The oracle as it stands: full periodic steps (retriangulation from
    scratch, forces, update) of the same workload from the state the timed
    region starts from, single thread."""
    import oracle

    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    n = len(xs)
    steps, t0 = 0, time.perf_counter()
    while True:
        xs, ys, th, _ = oracle.spv_run(xs, ys, th, Lx, Ly, P0, V0, 1, seed=1, step0=steps, dt=DT)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 50:
            break
    return {"value": n * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"{steps} full oracle steps of the N={n} workload (periodic Bowyer-Watson "
                      f"retriangulation + forces + update), {el:.1f} s, single thread"}


def batched_comparison(args, device):
    """512 independent replicas (N_r log-uniform on [256, 16384], p0 ~
    U[3.6, 4.0], v0 ~ U[0.01, 0.5], L_r = sqrt(N_r)), 2000 steps: all
    replicas in one context (one graph launch per step for all of them)
    versus one context per replica stepped in a loop (one graph launch per
    replica per step).  Both arms run the same first EQUIL_STEPS steps
    untimed; the fused arm then times every step of the rest of the 2000-step
    run (CUDA events around each step; 2 M cells hold ~2 GB of state, far
    more than L2) and the loop arm a window of steps right after the
    equilibration.  fused_over_loop compares the two on that same window."""
    import numpy as np
    import torch

    import paper_1702_02939_gb300 as cg
    import workloads

    R = 512
    total_steps = args.batched_steps
    sizes = workloads.replica_sizes(R, 7)
    p0s, v0s = workloads.replica_params(R, 7)
    reps, xs, ys, ths = [], [], [], []
    for r in range(R):
        x, y, th, L = workloads.spv_uniform(int(sizes[r]), 1000 + r)
        reps.append(dict(n=int(sizes[r]), Lx=L, Ly=L, p0=float(p0s[r]), v0=float(v0s[r])))
        xs.append(x); ys.append(y); ths.append(th)
    total = int(sizes.sum())
    stream = torch.cuda.current_stream()
    window = args.batched_window

    fused = cg.SPV(reps, np.concatenate(xs), np.concatenate(ys), np.concatenate(ths), dt=DT, seed=7,
                   device=device)
    fused.step(EQUIL_STEPS)
    launch, _ = fused.autotune(5, cache=launch_cache(args)) if not args.no_autotune else (fused.launch, None)
    timed = total_steps - EQUIL_STEPS
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(timed)]
    torch.cuda.synchronize()
    for k in range(timed):
        ev[k][0].record(stream)
        fused.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    fused.sync()
    per_step = [a.elapsed_time(b) for a, b in ev]
    fused.close()
    del fused
    singles = [cg.SPV([reps[r]], xs[r], ys[r], ths[r], dt=DT, seed=7, device=device) for r in range(R)]
    for sim in singles:
        sim.step(EQUIL_STEPS)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(window):
        for sim in singles:
            sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_l = e0.elapsed_time(e1)
    for sim in singles:
        sim.sync()
        sim.close()
    ms_fw = sum(per_step[:window])
    ms_f = sum(per_step)
    v_fw = total * window / (ms_fw * 1e-3)
    v_l = total * window / (ms_l * 1e-3)
    return {"workload": "spv_batched_R512_N256-16384_loguniform", "replicas": R, "cells": total,
            "run_steps": total_steps, "equilibration_steps": EQUIL_STEPS,
            "fused_cell_steps_per_s": total * timed / (ms_f * 1e-3), "fused_ms_per_step": ms_f / timed,
            "fused_timed_steps": [EQUIL_STEPS + 1, total_steps],
            "window_steps": [EQUIL_STEPS + 1, EQUIL_STEPS + window],
            "fused_window_cell_steps_per_s": v_fw, "per_replica_loop_cell_steps_per_s": v_l,
            "fused_over_loop": v_fw / v_l,
            "fused_window_ms_per_step": ms_fw / window, "loop_ms_per_step": ms_l / window,
            "fused_launch_shapes": launch}


def backward_cost(args, device):
    """Differentiable run: N = 4096, 1000 steps, checkpoint every 50, loss =
    mean over cells of (A (P/sqrt(A) - 3.95))^2 at the final state, per-cell p0
    ~ U[3.7, 3.9].  Times the checkpointed forward run and the reverse pass
    (which recomputes every segment) with CUDA events."""
    import numpy as np
    import torch

    import paper_1702_02939_gb300 as cg
    import workloads

    n, K, every = 4096, args.bwd_steps, 50
    x, y, th, L = workloads.spv_uniform(n, 3)
    sim = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=3.8, v0=0.1)], x, y, th, dt=DT, seed=11, device=device)
    sim.set_p0(np.random.default_rng(5).uniform(3.7, 3.9, n))
    sim.step(20)
    sim.sync()
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    bw = sim.run_checkpointed(K, every)
    e[1].record(stream)
    A, P = sim.geometry()
    r = P * A.sqrt() - 3.95 * A
    gA = 2.0 * r * (P / (2.0 * A.sqrt()) - 3.95) / n
    gP = 2.0 * r * A.sqrt() / n
    z = torch.zeros(n, dtype=torch.float64, device=device)
    torch.cuda.synchronize()
    e1b = torch.cuda.Event(enable_timing=True)
    e1b.record(stream)
    out = sim.backward(bw, K, every, z, z, gA, gP)
    e[2].record(stream)
    torch.cuda.synchronize()
    fwd_ms = e[0].elapsed_time(e[1])
    bwd_ms = e1b.elapsed_time(e[2])
    sim.close()
    return {"workload": "spv_grad_N4096_steps%d_ckpt%d" % (K, every), "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "backward_over_forward": bwd_ms / fwd_ms, "grad_KA": out[4], "grad_KP": out[5]}


def fp32_throughput(args, device):
    """The same SPV workload with single-precision physics (cg_params.precision
    = 1: FP32 geometry, forces and director terms; positions on the exact grid
    and exact topology): the 100 equilibration steps (and any extra warm-up)
    in FP64 (the random initial state's largest forces overflow FP32), 10 FP32
    steps, autotuned launch shapes, then each graph step timed alone with
    CUDA events, L2 flushed in between."""
    import torch

    import paper_1702_02939_gb300 as cg

    # the random initial state holds nearly coincident cells whose forces
    # overflow FP32; it is relaxed with FP64 steps first
    x, y, th, L = workload(args.n, 1)
    relax = cg.SPV([dict(n=args.n, Lx=L, Ly=L, p0=P0, v0=V0)], x, y, th, dt=DT, seed=1, device=device)
    relax.step(EQUIL_STEPS + args.warmup)
    x, y, th = relax.state()
    relax.close()
    del relax
    sim = cg.SPV([dict(n=args.n, Lx=L, Ly=L, p0=P0, v0=V0)], x, y, th, dt=DT, seed=1, precision="f32",
                 device=device)
    sim.set_step(EQUIL_STEPS + args.warmup)
    sim.step(10)
    sim.sync()
    launch, _ = (sim.autotune(10, flush_bytes=FLUSH_BYTES, cache=launch_cache(args)) if not args.no_autotune
                 else (sim.launch, None))
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    K = args.fp32_steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    ms = sum(a.elapsed_time(b) for a, b in ev) / K
    ph = sim.profile(20)
    sim.close()
    return {"workload": WORKLOAD.replace("fp64", "fp32"), "unit": UNIT, "dtype": "f32 physics, int64 grid, exact topology",
            "cell_steps_per_s": args.n / (ms * 1e-3), "ms_per_step": ms, "steps": K,
            "equilibration_steps": EQUIL_STEPS + args.warmup,
            "launch_shapes": launch, "phase_ms_per_step": {k: v / 20 for k, v in ph.items()}}


def avm_roofline(n, ph, prof_steps):
    """FP64 roofline of the dominant AVM kernel from its event-timed phase."""
    cells_ms = ph["cells_ms"] / prof_steps
    verts_ms = ph["vertices_ms"] / prof_steps
    if cells_ms >= verts_ms:
        kernel, flops, ms = "k_avm_cells", AVM_FLOPS["cells_per_cell"] * n, cells_ms
    else:
        kernel, flops, ms = "k_avm_force_move", AVM_FLOPS["vertices_per_vertex"] * 2 * n, verts_ms
    achieved = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": AVM_DRAM_BYTES_PER_LAUNCH.get(kernel),
            "duration_ms": ms,
            "note": "the kernel's own event-timed duration (eager launches); sqrt counts one flop but takes "
                    "an integer-pipe refinement; at N = 65536 the passes are latency bound"}


def decomposed_throughput(args, device):
    """One SPV system advanced as D strip domains in one process on this GPU
    (the domain decomposition's host protocol with its halo exchange after
    every step and a re-partition every 50 steps), against one context over
    the whole box from the same equilibrated state: cell-steps/s of both and
    whether their states agree bit for bit.  Timed on the host clock around
    synchronised runs (L2 not flushed)."""
    import numpy as np
    import torch

    import paper_1702_02939_gb300 as cg
    from paper_1702_02939_gb300 import domains

    n, D, steps = args.n, args.domains, args.domain_steps
    x, y, th, L = workload(n, 1)
    ref = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=P0, v0=V0)], x, y, th, dt=DT, seed=1, device=device)
    ref.step(EQUIL_STEPS)
    x0, y0, t0 = (t.cpu().numpy() for t in ref.state())
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    ref.step(steps)
    ref.sync()
    ms_ref = 1e3 * (time.perf_counter() - h0)
    rx, ry, rt = (t.cpu().numpy() for t in ref.state())
    ref.close()
    dd = domains.DecomposedSPV(x0, y0, t0, L, L, D, halo=8.0, p0=P0, v0=V0, repartition_every=50,
                               step0=EQUIL_STEPS, dt=DT, seed=1, device=device)
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    dd.step(steps)
    gx, gy, gt = dd.state()
    ms_dd = 1e3 * (time.perf_counter() - h0)
    halo = sum(len(p["ids"]) for p in dd.plans) - n
    dd.close()
    same = bool(np.array_equal(gx, rx) and np.array_equal(gy, ry) and np.array_equal(gt, rt))
    return {"workload": WORKLOAD, "domains": D, "steps": steps, "transport": "one process, one GPU",
            "halo_cells": int(halo), "undivided_cell_steps_per_s": n * steps / (ms_ref * 1e-3),
            "decomposed_cell_steps_per_s": n * steps / (ms_dd * 1e-3),
            "decomposed_ms_per_step": ms_dd / steps, "undivided_ms_per_step": ms_ref / steps,
            "bit_identical_to_undivided": same}


def avm_throughput(args, device):
    """Active vertex model (Sec. 2.D, Eq. 4, Fig. 1): N = 65536 cells (V =
    131072 vertices) from the Voronoi tessellation of uniform random seeds in
    L = 256, p0 = 3.8, v0 = 0.1, T1 threshold 0.04, dt = 0.01, FP64.  100
    equilibration steps, then each step (geometry, vertex force and move,
    directors, T1 passes) timed alone with CUDA events, L2 flushed in between.
    The oracle's AVM step from the initial network of the same seeds is timed
    beside it (one thread)."""
    import numpy as np
    import torch

    import oracle
    import paper_1702_02939_gb300 as cg
    import workloads

    n, thr, p0, v0 = 65536, 0.04, 3.8, 0.1
    x, y, th, L = workloads.spv_uniform(n, 21)
    sim = cg.AVM(n, L, L, x, y, th, p0=p0, v0=v0, dt=DT, t1_threshold=thr, seed=21, sort_every=AVM_SORT_EVERY,
                 device=device)
    sim.step(args.avm_warmup)
    sim.sync()
    c0 = sim.counters()
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    K = args.avm_steps  # 0: eager profiled steps only (no graph launch)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    c1 = sim.counters()
    # per step: cell pass, vertex pass, director terms, one kernel per T1
    # pass; per re-sort (after every AVM_SORT_EVERY-th step): 11 kernels
    sorts = (args.avm_warmup + K) // AVM_SORT_EVERY - args.avm_warmup // AVM_SORT_EVERY
    launches = 3 * K + (c1["loop_total"] - c0["loop_total"]) + 11 * sorts
    prof_steps = max(1, args.avm_profile_steps)
    ph = sim.profile(prof_steps)
    # oracle on the same kind of state (its own network build), a few steps
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    net = oracle.avm_build(xs, ys, Lx, Ly)
    oth, steps, t0 = th, 0, time.perf_counter()
    while True:
        net, oth, _ = oracle.avm_step(net, oth, p0, v0, seed=21, step=steps, dt=DT, thr=thr)
        steps += 1
        el = time.perf_counter() - t0
        if el > 5.0 or steps >= 200:
            break
    sim.close()
    V = 2 * n
    Kd = max(K, 1)
    return {"workload": "avm_N65536_L256_p0_3.8_v0_0.1_thr0.04_dt0.01_fp64", "unit": "vertex-steps/s",
            "vertex_steps_per_s": V * K / (ms * 1e-3) if K else None,
            "cell_steps_per_s": n * K / (ms * 1e-3) if K else None,
            "ms_per_step": ms / Kd if K else None, "steps": K, "warmup": args.avm_warmup, "l2": "flushed between timed steps",
            "sort_every": AVM_SORT_EVERY,
            "gpu_launches": launches,
            "t1_per_step": (c1["t1_total"] - c0["t1_total"]) / Kd,
            "t1_passes_per_step": (c1["t1_passes"] - c0["t1_passes"]) / Kd,
            "roofline": avm_roofline(n, ph, prof_steps),
            "phase_ms_per_step": {"cells": ph["cells_ms"] / prof_steps, "vertices": ph["vertices_ms"] / prof_steps,
                                  "directors": ph["dir_ms"] / prof_steps,
                                  "t1_passes": ph["t1_ms"] / prof_steps,
                                  "t1_passes_count": ph["t1_passes"] / prof_steps},
            "cpu_oracle": {"value": V * steps / el, "unit": "vertex-steps/s", "cores": 1, "kind": "oracle",
                           "sample": f"{steps} oracle AVM steps of the same N={n} network, {el:.1f} s"},
            "cell_death": avm_death_throughput(args, device)}


def avm_death_throughput(args, device):
    """The AVM workload with T2 transitions: 1% of the cells get A0 = 0 and
    are removed once they are triangles of area below 0.01 (T2 passes share
    the T1 passes).  After the same warm-up, each step is timed alone with
    CUDA events (L2 flushed in between) while the dying cells are removed."""
    import numpy as np
    import torch

    import paper_1702_02939_gb300 as cg
    import workloads

    if args.avm_steps == 0:  # profiled steps only
        return None
    n, thr, p0, v0 = 65536, 0.04, 3.8, 0.1
    x, y, th, L = workloads.spv_uniform(n, 21)
    cap = n + n // 50
    sim = cg.AVM(n, L, L, x, y, th, p0=p0, v0=v0, dt=DT, t1_threshold=thr, t2_area=0.01, seed=21, capacity=cap,
                 sort_every=AVM_SORT_EVERY, device=device)
    sim.step(args.avm_warmup)
    a0 = np.ones(cap)
    a0[np.random.default_rng(5).choice(n, n // 100, replace=False)] = 0.0
    sim.set_a0(a0)
    sim.sync()
    c0 = sim.counters()
    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    K = args.avm_steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    c1 = sim.counters()
    removed = int((sim.topology()[2][:n] == 0).sum())
    # divisions: 1% of the cells along random directions in one call (host
    # arrays in, outcome back; the call synchronizes), then the grown tissue steps
    rng = np.random.default_rng(6)
    alive = np.nonzero(sim.topology()[2].cpu().numpy() > 0)[0]
    cells = rng.choice(alive, n // 100, replace=False)
    ang = rng.uniform(0.0, np.pi, cells.size)
    dirs = np.stack([np.cos(ang), np.sin(ang)], 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    made = sim.divide(cells, dirs)
    div_s = time.perf_counter() - t0
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.zero_()
        ev2[k][0].record(stream)
        sim.step(1)
        ev2[k][1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    ms2 = sum(a.elapsed_time(b) for a, b in ev2)
    alive_after = int((sim.topology()[2] > 0).sum())
    sim.close()
    return {"workload": "avm_N65536_L256_p0_3.8_v0_0.1_thr0.04_t2area0.01_dying1pct_fp64", "unit": "vertex-steps/s",
            "vertex_steps_per_s": 2 * n * K / (ms * 1e-3), "ms_per_step": ms / K, "steps": K,
            "t2_per_step": (c1["t2_total"] - c0["t2_total"]) / K, "t1_per_step": (c1["t1_total"] - c0["t1_total"]) / K,
            "cells_removed": removed, "dying": n // 100,
            "divisions": {"requested": int(cells.size), "made": int(made.sum()), "call_ms": 1e3 * div_s,
                          "divisions_per_s": int(made.sum()) / div_s,
                          "ms_per_step_after": ms2 / K, "cells_alive_after": alive_after,
                          "cell_slots": cap}}


def sweep(args):
    """Time per step against system size and shape index, in the regimes of
    the paper's SPV timing figures: the solid regime (p0 = 3.8, v0 = 0.01,
    dt = 0.05; Fig. 2) and the fluid regime of the benchmark (p0 = 3.85,
    v0 = 0.1, dt = 0.01), N = 1024 ... 1048576; then p0 = 3.8 ... 4.0 at
    N = 65536, v0 = 0.1 (Fig. 3).  GPU: 100 warm-up steps, then 200 graph
    steps timed with CUDA events (default launch shapes).  CPU: the oracle's
    full periodic step, single thread, timed on the same state for N up to
    262144 (1 to 5 steps)."""
    import torch

    import __graft_entry__
    import oracle
    import paper_1702_02939_gb300 as cg
    import workloads

    __graft_entry__.build()
    stream = torch.cuda.current_stream()

    def gpu_time(n, p0, v0, dt, seed):
        x, y, th, L = workloads.spv_uniform(n, seed)
        sim = cg.SPV([dict(n=n, Lx=L, Ly=L, p0=p0, v0=v0)], x, y, th, dt=dt, seed=seed)
        sim.step(100)
        c0 = sim.counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(200)
        e1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        c1 = sim.counters()
        ms = e0.elapsed_time(e1) / 200
        xs, ys, ths = (t.cpu().numpy() for t in sim.state())
        sim.close()
        return ms, (c1["flagged_total"] - c0["flagged_total"]) / 200, (xs, ys, ths, L)

    def cpu_time(state, p0, v0, dt):
        xs, ys, ths, L = state
        Lx, Ly, q = oracle.box(L)
        xs, ys = oracle.snap_positions(xs, ys, Lx, Ly)
        steps, t0 = 0, time.perf_counter()
        while True:
            xs, ys, ths, _ = oracle.spv_run(xs, ys, ths, Lx, Ly, p0, v0, 1, seed=1, step0=steps, dt=dt)
            steps += 1
            el = time.perf_counter() - t0
            if el > 3.0 or steps >= 5:
                return 1e3 * el / steps

    rows = []
    regimes = {"solid": (3.8, 0.01, 0.05), "fluid": (3.85, 0.1, 0.01)}
    for name, (p0, v0, dt) in regimes.items():
        for n in (1024, 4096, 16384, 65536, 262144, 1048576):
            ms, flagged, state = gpu_time(n, p0, v0, dt, 5)
            cms = cpu_time(state, p0, v0, dt) if n <= 262144 else None
            rows.append({"regime": name, "n": n, "p0": p0, "v0": v0, "dt": dt, "gpu_ms_per_step": ms,
                         "cpu_oracle_ms_per_step": cms, "speedup": (cms / ms) if cms else None,
                         "flagged_per_step": flagged})
    for p0 in (3.8, 3.85, 3.9, 4.0):
        ms, flagged, state = gpu_time(65536, p0, 0.1, 0.01, 6)
        cms = cpu_time(state, p0, 0.1, 0.01)
        rows.append({"regime": "p0 scan", "n": 65536, "p0": p0, "v0": 0.1, "dt": 0.01, "gpu_ms_per_step": ms,
                     "cpu_oracle_ms_per_step": cms, "speedup": cms / ms, "flagged_per_step": flagged})
    # Hilbert re-sort period (Sec. 2.B), fluid regime at N = 262144
    sort_rows = []
    for every in (0, 10, 50, 200):
        x, y, th, L = workloads.spv_uniform(262144, 5)
        sim = cg.SPV([dict(n=262144, Lx=L, Ly=L, p0=3.85, v0=0.1)], x, y, th, dt=0.01, seed=5, sort_every=every)
        sim.step(100)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(400)
        e1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        sim.close()
        sort_rows.append({"sort_every": every, "gpu_ms_per_step": e0.elapsed_time(e1) / 400})
    # AVM time per step against N (Fig. 4), GPU and the AVM oracle
    avm_rows = []
    for n in (4096, 16384, 65536, 262144, 1048576):
        x, y, th, L = workloads.spv_uniform(n, 7)
        gms = {}
        for every in (0, AVM_SORT_EVERY):  # without and with the re-sort
            sim = cg.AVM(n, L, L, x, y, th, p0=3.8, v0=0.1, dt=0.01, t1_threshold=0.04, seed=7, sort_every=every)
            sim.step(50)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(200)
            e1.record(stream)
            torch.cuda.synchronize()
            sim.sync()
            sim.close()
            gms[every] = e0.elapsed_time(e1) / 200
        cms = None
        if n <= 262144:
            Lx, Ly, q = oracle.box(L)
            xs, ys = oracle.snap_positions(x, y, Lx, Ly)
            net = oracle.avm_build(xs, ys, Lx, Ly)
            oth, k, t0 = th, 0, time.perf_counter()
            while True:
                net, oth, _ = oracle.avm_step(net, oth, 3.8, 0.1, seed=7, step=k, thr=0.04)
                k += 1
                el = time.perf_counter() - t0
                if el > 2.0 or k >= 50:
                    break
            cms = 1e3 * el / k
        avm_rows.append({"n": n, "vertices": 2 * n, "gpu_ms_per_step": gms[AVM_SORT_EVERY],
                         "gpu_ms_per_step_unsorted": gms[0], "sort_every": AVM_SORT_EVERY,
                         "cpu_oracle_ms_per_step": cms, "ratio": (cms / gms[AVM_SORT_EVERY]) if cms else None})
    print(json.dumps({"study": "SPV time per step vs N and p0, Hilbert re-sort period, AVM vs N (GB300, FP64)",
                      "rows": rows, "sort_rows": sort_rows, "avm_rows": avm_rows}), flush=True)


def run_reference(args):
    """CPU oracle arm: each step is one oracle step of a spatial window of the
    N=262144 state, sized so that the whole run takes a few minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle

    x, y, th, L = workload(args.n, 1)
    Lx, Ly, q = oracle.box(L)
    xs, ys = oracle.snap_positions(x, y, Lx, Ly)
    n = len(xs)
    budget = 150.0 / max(1, args.steps + args.warmup)
    # calibrate the window half-width for about `budget` seconds per step
    hw = 8.0
    for _ in range(6):
        t0 = time.perf_counter()
        oracle.spv_window_step(xs, ys, th, Lx, Ly, P0, V0, 1, 0, Lx / 2, Ly / 2, hw)
        el = time.perf_counter() - t0
        if el > 0.5 * budget or hw >= Lx / 2 - 8:
            break
        hw = min(hw * 2.0, Lx / 2 - 8)
    scale = math.sqrt(max(budget / max(el, 1e-4), 0.05))
    hw = float(min(max(4.0, hw * scale), Lx / 2 - 8))
    rng = np.random.default_rng(0)
    total_cells, total_t, timed, skipped = 0, 0.0, 0, 0
    for s in range(args.warmup + args.steps):
        # every sample starts from the same state (the windows' updates are
        # not written back: a state patched window by window would develop
        # seams between moved and unmoved cells)
        cx = float(oracle.snap_length(rng.uniform(0, Lx), q))
        cy = float(oracle.snap_length(rng.uniform(0, Ly), q))
        for margin in (10.0, 16.0):
            try:
                t0 = time.perf_counter()
                _, _, _, k = oracle.spv_window_step(xs, ys, th, Lx, Ly, P0, V0, 1, s, cx, cy, hw, margin=margin)
                el = time.perf_counter() - t0
                break
            except oracle.OracleError:
                k = None
        if k is None:
            skipped += 1
            continue
        if s >= args.warmup:
            total_cells += k
            total_t += el
            timed += 1
    value = total_cells / total_t
    sample = (f"{timed} oracle steps of random square windows (half-width {hw:.1f}, ~{total_cells // max(timed, 1)} "
              f"cells updated each) of the N={n} initial state: exact triangulation of the window plus a "
              f"10-spacing margin, forces and update of its interior cells, single thread"
              + (f"; {skipped} windows skipped" if skipped else ""))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(timed, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_cells": n, "box": Lx, "sample": "window"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world)
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_1702_02939_gb300 as cg

    x, y, th, L = workload(args.n, 1 + rank)
    repair_cap = 4
    sim = cg.SPV([dict(n=args.n, Lx=L, Ly=L, p0=P0, v0=V0)], x, y, th, dt=DT, seed=1 + rank,
                 repair_cap=repair_cap, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    advance = sim.profile if args.eager else sim.step
    # the workload's equilibration, then the extra warm-up steps asked for;
    # then the launch shapes are tuned on a temporary copy of the state (the
    # simulation itself takes no step)
    advance(EQUIL_STEPS)
    advance(args.warmup)
    sim.sync()
    # tuned under the timing conditions of the timed region (L2 evicted before each step)
    launch, tune_ms = (sim.autotune(10, flush_bytes=FLUSH_BYTES, cache=launch_cache(args)) if not args.no_autotune
                       else (sim.launch, None))
    launch_source = "default" if args.no_autotune else ("stored" if tune_ms is None else "tuned")
    # the state the timed region starts from: the end-to-end run replays the same steps from it
    x0, y0, th0 = sim.state()
    step0 = sim.counters()["steps"]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    c_start = sim.counters()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()  # L2 flush (256 MB > 129 MB L2) between timed steps
        ev_s[k].record(stream)
        advance(1)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    sim.sync()  # raises on any device error
    ms = max_over_ranks(sum(ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)), world, "cuda")
    counters = sim.counters()
    value = weak_scaling_value(world, args.n, args.steps, ms)
    Kd = max(args.steps, 1)
    timed_state = {
        "equilibration_steps": EQUIL_STEPS, "extra_warmup_steps": args.warmup,
        "first_timed_step": step0 + 1, "last_timed_step": counters["steps"],
        "flagged_cells_per_step": (counters["flagged_total"] - c_start["flagged_total"]) / Kd,
        "repaired_cells_per_step": (counters["repaired_total"] - c_start["repaired_total"]) / Kd,
        "repair_rounds_per_step": (counters["loop_total"] - c_start["loop_total"]) / Kd,
        "last_flagged": counters["last_flagged"]}

    # per-kernel device times (eager launches, CUDA events on the same stream)
    prof_steps = max(1, args.avm_profile_steps)
    ph = sim.profile(prof_steps)
    dominant = max(("geometry", "force_move"), key=lambda k: ph[k])
    dom_ms = ph[dominant] / prof_steps
    achieved_tflops = FLOPS_PER_CELL[dominant] * args.n / (dom_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                "traffic": GEOM_DRAM_BYTES_PER_LAUNCH if dominant == "geometry" else None,
                "kernel": {"geometry": "k_geom", "force_move": "k_force"}[dominant], "duration_ms": dom_ms,
                "peak_source": "FP64 nominal from unit counts x 2.07 GHz (FP64 units, not tensor)"}
    hbm_gbs, hbm_src = hbm_peak()
    step_s = ms * 1e-3 / args.steps
    hbm = {"achieved_gbs": BYTES_PER_CELL_STEP * args.n / step_s / 1e9, "peak_gbs": hbm_gbs,
           "frac": BYTES_PER_CELL_STEP * args.n / step_s / 1e9 / hbm_gbs, "source": hbm_src,
           "bytes_per_cell_step": BYTES_PER_CELL_STEP}

    # end to end through the public API with pinned host buffers, over the
    # same steps from the same state as the timed region: every step uploads
    # that step's per-cell v0 and reads back the positions.  Each step is one
    # cg_run_io call after the same L2 flush as the timed region (host clock,
    # flush excluded); the pipelined figure runs the steps in one call, the
    # copies of one step overlapping the kernels of the next (L2 not flushed).
    e2e = None
    if not args.no_e2e:
        hv0 = torch.full((args.n,), V0, dtype=torch.float64).pin_memory()
        hx = torch.empty(args.n, dtype=torch.float64).pin_memory()
        hy = torch.empty(args.n, dtype=torch.float64).pin_memory()

        def restore():
            sim.set_state(x0, y0, th0)
            sim.set_step(step0)
            sim.sync()

        restore()
        el = 0.0
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.run_io(1, v0=hv0, x=hx, y=hy)
            el += time.perf_counter() - t0
        el = max_over_ranks(el, world, "cuda")
        same = sim.counters()["steps"] == counters["steps"]
        restore()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.run_io(args.steps, v0=hv0, x=hx, y=hy)
        elp = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": weak_scaling_value(world, args.n, args.steps, 1e3 * el), "unit": UNIT,
               "h2d_bytes_per_step": 8 * args.n, "d2h_bytes_per_step": 16 * args.n,
               "api": "cg_run_io, one call per step (v0 uploaded from pinned host memory, positions downloaded "
                      "to pinned host memory), host clock",
               "steps": args.steps, "same_steps_as_timed_region": bool(same),
               "l2": "flushed before every step, as the timed region (flush not timed)",
               "pipelined": {"value": weak_scaling_value(world, args.n, args.steps, 1e3 * elp), "unit": UNIT,
                             "api": "cg_run_io, all steps in one call: copies on two copy streams overlap the "
                                    "kernels of neighbouring steps", "l2": "not flushed"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(x0.cpu().numpy(), y0.cpu().numpy(), th0.cpu().numpy(), L, args.cpu_seconds)
    sim.close()
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = batched_comparison(args, f"cuda:{local}")
    backward = None
    if rank == 0 and world == 1 and not args.no_backward:
        backward = backward_cost(args, f"cuda:{local}")
    decomposed = None
    if rank == 0 and world == 1 and args.domains >= 2:
        decomposed = decomposed_throughput(args, f"cuda:{local}")
    avm = None
    if rank == 0 and world == 1 and not args.no_avm:
        avm = avm_throughput(args, f"cuda:{local}")
    fp32 = None
    if rank == 0 and world == 1 and not args.no_fp32:
        fp32 = fp32_throughput(args, f"cuda:{local}")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n_cells": args.n, "box": L, "p0": P0, "v0": V0, "dt": DT,
                           "equilibration_steps": EQUIL_STEPS,
                           "replicas_per_gpu": 1, "l2": "flushed between timed steps (256 MB write)",
                           "repair_cap": repair_cap, "launch": "eager" if args.eager else "graph",
                           "launch_shapes": launch, "launch_source": launch_source,
                           "autotune_ms_per_step": tune_ms},
                "clocks": clk, "e2e": e2e,
                "gpu_launches": (kernels_launched(args.steps, args.steps * repair_cap, True, launch["ring_order"])
                                 if args.eager else
                                 kernels_launched(args.steps, counters["loop_total"] - c_start["loop_total"], False,
                                                  launch["ring_order"], launch.get("force_beside", 0))),
                "timed_state": timed_state,
                "roofline": roofline, "hbm_roofline": hbm, "cpu_baseline": cpu,
                "phase_ms_per_step": {k: v / prof_steps for k, v in ph.items()},
                "counters": counters, "batched": batched, "backward": backward, "avm": avm, "fp32": fp32,
                "decomposed": decomposed}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.sweep:
        sweep(args)
        return
    if args.avm_only:
        import __graft_entry__

        __graft_entry__.build()
        print(json.dumps(avm_throughput(args, "cuda:0")), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
