"""The N > 1 path of bench.py on CPU: replicas on world_size 2 gloo ranks take the max of their timed regions over
ranks (max_over_ranks) and report the units all ranks processed per second of the slowest (whole_job_rate)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, seconds, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(seconds[rank], "cpu")
        dist.barrier()
        out[rank] = (m, bench.whole_job_rate(6.0, world, m))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    world, seconds = 2, [1.5, 2.0]
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), seconds, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        m, v = out[r]
        assert m == 2.0                 # the slowest rank's timed region
        assert v == 6.0 * world / 2.0   # 6 units per rank, both ranks, over the slowest time


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(10.0, 1, 4.0) == 2.5
