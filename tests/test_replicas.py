"""Replicas on several GPUs: the bench's only collective is the timing maximum
(world size 2 over gloo on the CPU; no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


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
        t_max = bench.max_over_ranks(times[rank])
        out[rank] = (t_max, bench.replica_throughput(129 * 3, world, t_max))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput():
    world, port = 2, _free_port()
    times = [1000.0, 1250.0]  # ms of the timed region on each rank
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t_max, value = res[r]
        assert t_max == 1250.0
        assert value == pytest.approx(129 * 3 * 2 / 1.25)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.replica_throughput(10, 1, 2000.0) == pytest.approx(5.0)
