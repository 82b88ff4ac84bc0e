"""Multi-rank bench logic on CPU (gloo, world size 2): every rank sorts its
own instance (weak scaling, no collective on the data path); the reported
time is the slowest rank's and the value counts all ranks' keys."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 20.0][rank]
    slowest = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.whole_job_gkeys(1 << 28, world, slowest)
    dist.barrier()
    out[rank] = (slowest, value)
    dist.destroy_process_group()


def test_weak_scaling_reports_slowest_rank_and_all_keys():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        slowest, value = out[rank]
        assert slowest == 20.0
        assert value == pytest.approx((1 << 28) * 2 / 0.020 / 1e9)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.whole_job_gkeys(1 << 20, 1, 1.0) == pytest.approx((1 << 20) / 1e-3 / 1e9)
