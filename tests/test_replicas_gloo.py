"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path does not shard: N ranks run N independent replicas of the same
matrix-vector product, with a barrier around the timed steps and the job's
time taken as the slowest rank's.  These tests run that aggregation over a
real two-process gloo group, and the reference arm's rule that ranks other
than 0 do no work.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import bench
    dist = bench.init_ranks(world, backend="gloo")
    try:
        ms = 10.0 + 5.0 * rank                    # rank 1 is the slow replica
        dist.barrier()
        m = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        v = bench.replica_value(world, 1000 * 1000, m)
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_value_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in got:
        assert m == 15.0                           # every rank sees the slowest time
        assert v == pytest.approx(2 * 1e6 / 15e-3)  # N replicas' work over that time


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.init_ranks(1) is None
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.replica_value(1, 4e6, 2.0) == pytest.approx(2e9)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import argparse
    import bench
    from paper_1902_05875_gb300 import workloads as W
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: called.append(1))
    args = argparse.Namespace(gpus=2, steps=1, warmup=1)
    bench.run_reference(args, W.cfg_small())
    assert called == [] and capsys.readouterr().out == ""
