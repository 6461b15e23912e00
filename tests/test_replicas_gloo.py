"""The N > 1 path of bench.py on the CPU: independent replicas, one per rank, whose
timings are combined by a max over the ranks (gloo, world size 2) and whose work adds
up; no collective touches the data path."""
import os
import socket

import pytest
import torch.multiprocessing as mp


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
    # rank r pretends its device time was 1 + r s and its wall time 10 - r s
    dev, wall = bench.max_over_ranks(dist, [1.0 + rank, 10.0 - rank], "cpu")
    out[rank] = (dev, wall, bench.job_throughput(world, 1000.0, 4, dev))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        dev, wall, v = out[r]
        assert dev == 2.0 and wall == 10.0
        assert v == pytest.approx(world * 1000.0 * 4 / 2.0)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.job_throughput(1, 10.0, 5, 2.0) == 25.0
