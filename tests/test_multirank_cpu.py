"""The multi-GPU benchmark path on CPU: two gloo ranks, each with its own DM-trial batch (weak
scaling, no data-path collective), a barrier around the timed region and the slowest rank's time
taken as the step time."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    seed, offsets, _ = bench.rank_workload(64, rank)
    bench.barrier(world)
    slowest = bench.reduce_max(float(10 + rank), world)
    total = int(offsets[-1])
    tot = [None] * world
    dist.all_gather_object(tot, total)
    q.put((rank, seed, total, slowest, sum(tot)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, m0, all0), (r1, s1, t1, m1, all1) = res
    assert s0 != s1  # each rank has its own batch
    assert m0 == m1 == 11.0  # both ranks see the slowest rank's time
    assert all0 == all1 == t0 + t1  # whole-job bins = sum over ranks
