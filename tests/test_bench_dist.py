"""The multi-rank path of bench.py on the CPU: two gloo ranks, max-over-ranks
timing and whole-job units (each rank is an independent replica)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r) == (world, rank)
    agg = bench.aggregate(1.0 + rank, 5, world)
    bench.barrier(world)
    q.put((rank, agg))
    dist.destroy_process_group()


def test_two_rank_aggregate_is_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r]["max_seconds"] == 2.0
        assert res[r]["total_units"] == 10
        assert abs(res[r]["seconds_per_unit"] - 0.2) < 1e-12
