"""The bench's multi-rank path on the CPU: two gloo ranks (one replica of the workload each,
weak scaling) combine their timings as the slowest rank's time and their work as the sum,
which is what `bench.py --gpus N` reports under torchrun."""
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


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.reduce_over_ranks(torch, dist, world, "cpu", ms=10.0 + rank, work=100.0 * (rank + 1))
    dist.barrier()
    out.put((rank, ms, work))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 11.0, 300.0), (1, 11.0, 300.0)]


def test_single_process_passes_values_through():
    import bench
    assert bench.reduce_over_ranks(torch, None, 1, "cpu", 3.5, 7.0) == (3.5, 7.0)
