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


def _rank_executor(rank, world, port, out):
    """One replica: this rank's own executor (a dry-run context: chains are analysed and
    planned, nothing runs on a device) flushes the same chain `steps` times."""
    import time

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1709_02125_gb300 import oc
    from workloads import random_chain
    oc.load()
    n, steps = 512, 3
    dats, reds, loops = random_chain.build(n=n, dtype="f32")
    for d in dats:
        d.init = None
    fp = random_chain.footprint_bytes(n, 24, 4)
    with oc.Executor(fp // 3, dryrun=True, flags=oc.OC_FLAG_PREFETCH | oc.OC_FLAG_CYCLIC) as ex:
        for d in dats:
            ex.decl_dat(d)
        for r in reds:
            ex.decl_reduction(r.name, r.op)
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            for lp in loops:
                ex.enqueue(lp)
            ex.flush()
        secs = time.perf_counter() - t0
        st = ex.stats()
    (t,) = bench.max_over_ranks(dist, [secs], "cpu")
    per_step = st["total_cell_updates"] / steps
    out[rank] = (st["tiles"], st["tile_height"], st["chains"], per_step, secs, t,
                 bench.job_throughput(world, per_step, steps, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_drive_their_own_executors():
    import __graft_entry__
    __graft_entry__.build_lib()
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_executor, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    # the same chain gives the same plan and the same work on every replica
    assert r0[:4] == r1[:4] and r0[0] > 1 and r0[2] == 3
    # the job's time is the slowest replica's; its work is every replica's
    assert r0[5] == r1[5] == max(r0[4], r1[4])
    assert r0[6] == pytest.approx(world * r0[3] * 3 / r0[5])
