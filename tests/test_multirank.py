"""Multi-rank path of the bench on CPU: beams are independent replicas, so the only
cross-rank step is the max over ranks of the timings (gloo, world size 2)."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0 + 5.0 * rank, 30.0 - rank]          # rank 1 is slower on the first timer
    got = bench.reduce_max(ms, dist)
    rate = bench.whole_job_rate(1000.0, 4, world, got[0])
    out[rank] = (got, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_and_rate_two_ranks():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    for r in range(world):
        got, rate = out[r]
        assert got == [15.0, 30.0]
        assert rate == pytest.approx(1000.0 * 4 * 2 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max([1.5, 2.5]) == [1.5, 2.5]
    assert bench.whole_job_rate(10.0, 2, 1, 1000.0) == 20.0
