"""The bench's multi-rank path (independent replicas) on CPU: two gloo ranks, no GPU.

Each rank times its own circuit; the reported time is the maximum over ranks and the value is
every rank's units over that time.  Rendezvous on 127.0.0.1.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, device="cpu")
    value = bench.whole_job_rate(1e9, world, ms_max / 1e3)
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_max_time_and_whole_job_rate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0] == out[1]
    ms_max, value = out[0]
    assert ms_max == 150.0
    assert value == pytest.approx(2e9 / 0.150)


def test_single_rank_without_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
