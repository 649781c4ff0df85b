"""Multi-GPU host logic, checked with gloo ranks on the CPU (no GPU needed).

* Replicas of one system (the default benchmark under torchrun): the timed region is the
  slowest rank's, and the per-iteration time is NOT divided by the number of GPUs (a replica
  does not make any system iterate faster); the job's rate is reported separately.
* Batches of independent systems: partitioned across ranks by their o^2 v^4, every system on
  exactly one rank, loads balanced; the per-system results reach every rank, in batch order,
  through one all_gather.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_rank(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(times[rank], device="cpu")
        out[rank] = (ms, bench.seconds_per_step(ms, 4), bench.replica_throughput(ms, 4, world)["steps_per_s"])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_do_not_divide_the_iteration_time():
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    times = [120.0, 200.0]  # ms of the timed region on each rank
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that already runs threads
        out = m.dict()
        mp.spawn(_replica_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value, rate = res[r]
        assert ms == 200.0
        assert value == pytest.approx(200.0 / 1e3 / 4)
        assert rate == pytest.approx(2 * 4 / 0.2)


def test_single_process_is_unchanged():
    import bench
    assert bench.max_over_ranks(75.0, device="cpu") == 75.0
    assert bench.seconds_per_step(75.0, 5) == pytest.approx(0.015)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_system_once_and_balances_the_ladder_cost(world):
    from paper_2103_08473_gb300 import inputs, shard
    shapes = inputs.batch_shapes(64, 4)
    costs = [shard.ladder_cost(o, v) for (o, v, _, _) in shapes]
    parts = shard.partition(costs, world)
    assert len(parts) == world
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(64))
    assert all(p == sorted(p) for p in parts)
    loads = [sum(costs[k] for k in p) for p in parts]
    mean = sum(costs) / world
    # longest-processing-time bound: no rank exceeds the mean by more than the largest system
    assert max(loads) <= mean + max(costs)
    if world <= 4:
        assert max(loads) / min(loads) < 1.1


def test_partition_is_deterministic_and_rejects_bad_world():
    from paper_2103_08473_gb300 import shard
    costs = [5.0, 5.0, 3.0, 1.0, 1.0]
    assert shard.partition(costs, 2) == shard.partition(costs, 2) == [[0, 2], [1, 3, 4]]
    with pytest.raises(ValueError):
        shard.partition(costs, 0)


def _gather_rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_2103_08473_gb300 import inputs, shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shapes = inputs.batch_shapes(64, 4)
        parts = shard.partition([shard.ladder_cost(o, v) for (o, v, _, _) in shapes], world)
        # fake per-system results that name their system and the rank that produced them
        rows = {k: [float(k), -0.5 * k, float(rank), float(shapes[k][0])] for k in parts[rank]}
        out[rank] = (shard.gather_results(rows, 64, 4), parts)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_every_systems_result_in_batch_order():
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_gather_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    from paper_2103_08473_gb300 import inputs
    shapes = inputs.batch_shapes(64, 4)
    t0, parts = res[0]
    for r in range(world):
        np.testing.assert_array_equal(res[r][0], t0)  # every rank sees the same table
    np.testing.assert_array_equal(t0[:, 0], np.arange(64))
    np.testing.assert_array_equal(t0[:, 1], -0.5 * np.arange(64))
    np.testing.assert_array_equal(t0[:, 3], [s[0] for s in shapes])
    for r, p in enumerate(parts):
        assert np.all(t0[p, 2] == r)


def test_gather_without_a_process_group_returns_the_local_rows():
    from paper_2103_08473_gb300 import shard
    t = shard.gather_results({1: [2.0, 3.0]}, 3, 2)
    assert t[1].tolist() == [2.0, 3.0] and np.all(np.isnan(t[[0, 2]]))
