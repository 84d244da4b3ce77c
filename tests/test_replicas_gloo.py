"""Multi-GPU runs are independent replicas: the only cross-rank step is the maximum of the per-rank
timings. Exercised here with two gloo ranks on the CPU (no GPU needed)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = [10.0 + rank, 100.0 - 7 * rank]  # this rank's step and end-to-end milliseconds
    out[rank] = bench.max_over_ranks(local, world)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == [11.0, 100.0]


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([3.5, 2.0], 1) == [3.5, 2.0]
