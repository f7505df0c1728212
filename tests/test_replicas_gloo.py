"""The multi-GPU path of the bench is independent replicas (the solve does
not shard): a barrier before the timed solves, each replica's total time,
the MAX over ranks, and value = world x steps / max.  Checked here with two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TIMES = {0: [1.0, 2.0, 0.5], 1: [1.5, 1.6, 0.4]}    # seconds per timed solve, per rank


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, REPO)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        q.put((rank, *bench.aggregate_replicas(TIMES[rank], world)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    slowest = max(sum(v) for v in TIMES.values())
    for rank, value, total_max in got:
        assert total_max == pytest.approx(slowest)
        assert value == pytest.approx(2 * 3 / slowest)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, REPO)
    import bench
    value, total = bench.aggregate_replicas([0.5, 0.25], 1)
    assert total == pytest.approx(0.75) and value == pytest.approx(2 / 0.75)
