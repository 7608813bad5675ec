"""The multi-rank bench logic (replicas, max-over-ranks timing) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank                 # rank 1 is the slow one
        got = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (got, bench.job_rate(world, 20 * 5, got))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:      # no fork from a process that may hold threads
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # whole-job rate: units of both ranks over the slowest rank's time
    assert res[0][1] == pytest.approx(2 * 100 * 1000.0 / 150.0)


def test_single_process_is_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_rate(1, 20, 1000.0) == pytest.approx(20.0)
