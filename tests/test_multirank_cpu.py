"""The N > 1 bench path on CPU: two gloo ranks (one process each, no GPU)
combine their per-rank step time and work the way bench.py does under
torchrun -- the slowest rank's time, the sum of the work (weak scaling, no
data-path collective) -- and every rank gets the same whole-job numbers."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: a step of 10 + 5 r ms over 1e12 (r + 1) bit operations
        ms, value = bench.job_line_values(10.0 + 5.0 * rank, 1e12 * (rank + 1), dist, torch.device("cpu"))
        assert bench.reduce_over_ranks(float(rank), "max", dist, torch.device("cpu")) == world - 1
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_same_whole_job_numbers():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
    expect_ms = 15.0                          # the slower rank
    expect_value = 3e12 / (expect_ms / 1000)  # the work of both
    for r in range(world):
        ms, value = out[r]
        assert ms == pytest.approx(expect_ms)
        assert value == pytest.approx(expect_value)


def test_one_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_line_values(20.0, 2e12, None, None)
    assert ms == 20.0 and value == pytest.approx(1e14)
