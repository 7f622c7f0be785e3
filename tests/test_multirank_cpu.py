"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
simulates its own frame, so the only exchange is the timing reduction, which
must give every rank the slowest rank's time and count all ranks' beams."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [30.0, 50.0][rank]  # 3 steps, rank 1 is slower
    rate, ms = bench.job_rate(local_ms, 1000, 3, world, dist)
    dist.barrier()
    out[rank] = (rate, ms)
    dist.destroy_process_group()


def test_job_rate_takes_slowest_rank_and_counts_all_beams():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        rate, ms = out[r]
        assert ms == pytest.approx(50.0 / 3)
        assert rate == pytest.approx(world * 1000 / (50.0 / 3 * 1e-3))


def test_job_rate_single_rank():
    import bench
    rate, ms = bench.job_rate(20.0, 500, 4, 1)
    assert ms == pytest.approx(5.0) and rate == pytest.approx(500 / 5e-3)
