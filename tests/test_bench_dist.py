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


def test_reference_arm_line_keeps_the_contract(monkeypatch):
    """bench.py --impl reference on the CPU (the oracle as the reference arm): rank 0
    prints the JSON line with the contract's keys; other ranks do no work.  Run on a
    small lattice so that the test takes a second."""
    import argparse
    import bench
    monkeypatch.setattr(bench, "L_FINE", (4, 4, 4, 4))
    monkeypatch.setattr(bench, "LS", 8)
    args = argparse.Namespace(steps=2, warmup=1, gpus=1, impl="reference", workload="two-level")
    assert bench.run_reference(args, 2, 1) is None
    line = bench.run_reference(args, 1, 0)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "dtype",
              "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["higher_is_better"] is False
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert "workload" in line["config"]
