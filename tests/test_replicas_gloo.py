"""The multi-rank bench path (independent replicas, weak scaling) on CPU:
two gloo ranks, the step time is the slowest rank's and the throughput counts
every rank's targets.  No GPU and no data-path collective is involved."""
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


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(1.5 + rank, dist, "cpu")  # rank 1 is slower
    out[rank] = (ms, bench.job_throughput(1000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == pytest.approx(2 * 1000 / 2.5e-3)


def test_single_rank_is_unchanged():
    import bench

    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.job_throughput(10, 1, 2.0) == pytest.approx(5000.0)
