"""The N > 1 path of bench.py on CPU: independent replicas, a barrier and a
max-over-ranks timing reduction over world_size-2 gloo ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, ms_values, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    dist.barrier()
    ms = bench.replica_max_ms(ms_values[rank], dist)
    out[rank] = ms
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ms_values = [120.0, 150.5]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), ms_values, out), nprocs=2, join=True,
                       start_method="spawn")
    assert out[0] == out[1] == 150.5
    v = bench.replica_value(64, out[0], 2)
    assert v == pytest.approx(2 * 64 / 0.1505)


def test_single_rank_needs_no_collective():
    assert bench.replica_max_ms(12.5, None) == 12.5
    assert bench.replica_value(10, 1000.0, 1) == pytest.approx(10.0)
