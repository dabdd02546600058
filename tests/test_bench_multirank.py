"""The N>1 path of bench.py runs independent replicas (one problem per GPU, no
data-path exchange) and reports the whole job at the pace of its slowest
rank. Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]                     # the second replica is slower
    m = bench.max_over_ranks(ms)
    out[rank] = bench.job_throughput(world, 10, m)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_at_the_slowest_pace():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == out[1] == pytest.approx(2 * 10 / 0.150)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 4, 2000.0) == pytest.approx(2.0)
