"""The multi-replica (N > 1) timing of bench.py on CPU ranks: two gloo
processes, each with its own timed region; every rank must see the slowest
replica's time and the job rate must count the units of all replicas."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total = bench.replica_total(1.0 + 0.5 * rank, world, "cpu")
    out[rank] = (total, bench.job_rate(5, world, total))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_units():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        total, rate = res[rank]
        assert total == 1.5               # the slower replica
        assert rate == 5 * world / 1.5    # units of both replicas over the job time


def test_one_replica_is_unchanged():
    import bench
    assert bench.replica_total(2.5, 1, "cpu") == 2.5
    assert bench.job_rate(4, 1, 2.0) == 2.0
