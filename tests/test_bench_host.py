"""Host-side logic of bench.py: bond-dimension schedule, flop counts and the
multi-rank aggregation (max time, summed solves), the latter over two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_schedule_and_flops():
    s = bench.schedule(4, 64, 30)
    assert s[:5] == [(4, 4, 16), (4, 16, 16), (16, 16, 64), (16, 64, 64), (64, 64, 64)]
    assert all(x == (64, 64, 64) for x in s[4:])
    s2 = bench.schedule(2, 64, 8)
    assert s2[:7] == [(2, 2, 4), (2, 4, 4), (4, 4, 16), (4, 16, 16), (16, 16, 64), (16, 64, 64),
                      (64, 64, 64)]
    f = bench.step_flops(64, 64, 64)
    assert f["s2"] == 2 * 64 ** 7
    assert f["total"] == 2 * 64 ** 7 + 4 * 64 ** 6 + 6 * 64 ** 6 - 4 * 64 ** 6 + 4 * 64 ** 6
    assert bench.products_of_step(5, 5, 2, "bf16x6") == 10
    assert bench.products_of_step(7, 5, 2, "bf16x6") == 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, solves = bench.aggregate_over_ranks(100.0 + 50.0 * rank, 3, dist, torch.device("cpu"))
    out[rank] = (ms, solves)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (150.0, 6.0) and out[1] == (150.0, 6.0)


def test_aggregate_single_rank():
    assert bench.aggregate_over_ranks(12.5, 3) == (12.5, 3)
