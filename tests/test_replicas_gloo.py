"""The benchmark's multi-GPU path is replicas only (each rank builds its own
copy; no exchange on the data path).  Its host logic -- the max-over-ranks
time and the whole-job throughput -- runs here as world-size-2 gloo ranks on
the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank              # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, dist, device="cpu")
        out[rank] = (worst, bench.replica_throughput(1000.0, worst, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of a threaded test process
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    worst, thr = out[0]
    assert worst == 15.0
    assert thr == pytest.approx(2 * 1000.0 / 0.015)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.replica_throughput(10.0, 1000.0, 1) == pytest.approx(10.0)
