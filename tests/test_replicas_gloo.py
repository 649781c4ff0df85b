"""The multi-GPU form of the benchmark is replicas (every rank runs the whole workload, no
data-path collective): its timing takes the slowest rank and reports the whole job's seconds
per iteration. Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], device="cpu")
        out[rank] = (ms, bench.whole_job_seconds_per_iteration(ms, 4, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    times = [120.0, 200.0]  # ms of the timed region on each rank
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that already runs threads
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 200.0
        assert value == pytest.approx(200.0 / 1e3 / 4 / 2)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(75.0, device="cpu") == 75.0
    assert bench.whole_job_seconds_per_iteration(75.0, 5, 1) == pytest.approx(0.015)
