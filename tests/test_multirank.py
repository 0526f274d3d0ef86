"""Host logic of the multi-rank bench (weak-scaling replicas) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
        out[rank] = (ms, bench.whole_job_value(world, 1024, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_all_elements():
    world, port = 2, _free_port()
    times = [1000.0, 2500.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == pytest.approx(2500.0)
        assert value == pytest.approx(2 * 1024 / 2.5)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.whole_job_value(1, 1024, 500.0) == pytest.approx(2048.0)
