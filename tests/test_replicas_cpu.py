"""The multi-GPU mode of bench.py runs independent replicas (one per rank, no
collective on the data path): its only exchange is the maximum of the ranks'
timed totals.  Checked here with two gloo ranks on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1200.0, 1500.0][rank]
    value, tot = bench.replica_throughput(local_ms, 10, world, "cpu")
    out[rank] = (value, tot)
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, tot = out[r]
        assert tot == 1500.0
        assert value == pytest.approx(world * 10 / 1.5)


def test_one_replica_needs_no_process_group():
    import bench
    value, tot = bench.replica_throughput(500.0, 4, 1)
    assert (value, tot) == (8.0, 500.0)
