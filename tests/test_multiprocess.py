"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The SPV step does not shard (replicas only): each rank advances its own
system and the job reports the slowest rank's time and the summed
throughput.  These tests run that reduction with two gloo ranks on CPU.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, w, "cpu")
    value = bench.weak_scaling_value(w, 1000, 4, ms)
    dist.barrier()
    results.put((r, w, local, ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_summed_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, results)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(results.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, local, ms, value) in enumerate(out):
        assert (r, w, local) == (rank, world, rank)
        assert ms == 15.0  # the slowest rank's time on every rank
        assert value == pytest.approx(world * 1000 * 4 / 15e-3)


def test_one_rank_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.weak_scaling_value(1, 262144, 1000, 400.0) == pytest.approx(262144 * 1000 / 0.4)
