"""The multi-rank path of bench.py (one independent box per rank, replicas):
with two gloo ranks on the CPU, every rank sees the slowest rank's time and
the whole-job rate counts all ranks' work over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [120.0, 150.0][rank]  # rank 1 is the slowest
    slow = bench.slowest(tdist, local_ms, "cpu")
    rate = bench.job_rate(ws, 3_000_000 * 100, slow / 1e3)
    tdist.barrier()
    tdist.destroy_process_group()
    out[rank] = (slow, rate)


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] == pytest.approx(2 * 3_000_000 * 100 / 0.150)
    assert out[0][1] == out[1][1]


def test_single_rank_needs_no_group():
    assert bench.slowest(None, 7.5, "cpu") == 7.5
    assert bench.job_rate(1, 1000, 2.0) == 500.0
