"""The bench's multi-rank logic on CPU: two gloo ranks, each timing its own
replica; the job's time is the slowest rank's and its rate counts every
rank's updates."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = 10.0 + 5.0 * rank  # rank 1 is the slow one
    got = bench.max_over_ranks(torch, mine, dist, torch.device("cpu"))
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_whole_job_rate_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.whole_job_rate(1, 4096.0 * 4096.0, 1000, 5, 50.0)
    two = bench.whole_job_rate(2, 4096.0 * 4096.0, 1000, 5, 50.0)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(4096.0 * 4096.0 * 1000 * 5 / 0.05 / 1e9)


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import torch
    import bench
    assert bench.max_over_ranks(torch, 3.5, None, None) == 3.5
