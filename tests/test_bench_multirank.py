"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
GPU in a real run) reduce their timings to the slowest rank's, and the
whole-job throughput counts the units of every rank over that time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, w, dist = bench.dist_setup(world, backend="gloo")
    assert (r, w) == (rank, world)
    bench.barrier(dist)
    slowest = bench.max_over_ranks(0.5 + rank, dist)   # rank 1 is the slow one
    value = bench.job_throughput(1000, 10, w, slowest)
    out[rank] = (slowest, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    world = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    slowest, value = out[0]
    assert slowest == 1.5
    assert value == pytest.approx(1000 * 10 * 2 / 1.5)
