"""Multi-rank host logic of bench.py (replicas, max-over-ranks timing) on
CPU with the gloo backend, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [2.0, 3.0][rank]
    worst = bench.max_over_ranks(local_seconds, world, "cpu")
    value = bench.job_mlups(1000, 10, world, worst)
    dist.barrier()
    out[rank] = (worst, value)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        worst, value = out[r]
        assert worst == 3.0
        assert value == pytest.approx(world * 1000 * 10 / 3.0 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.job_mlups(4096 * 4096, 2000, 1, 1.0) == pytest.approx(4096 * 4096 * 2000 / 1e6)
