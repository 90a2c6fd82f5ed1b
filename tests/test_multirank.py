"""The benchmark's multi-rank host logic on CPU with two gloo ranks: each
rank is an independent replica, the job time is the slowest rank's, and the
job throughput counts every rank's units."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [2.0, 5.0][rank]          # rank 1 is the slowest
    rate, ms = bench.job_rate(local_ms, 1000, world, dist, "cpu")
    out[rank] = (rate, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:   # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        rate, ms = res[rank]
        assert ms == 5.0                        # MAX over ranks
        assert rate == pytest.approx(2 * 1000 / 5e-3)


def test_job_rate_single_rank():
    import bench
    rate, ms = bench.job_rate(4.0, 100, 1)
    assert ms == 4.0 and rate == pytest.approx(100 / 4e-3)
