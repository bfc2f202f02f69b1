"""The multi-GPU path is replicas only: every logL is independent, so each rank
evaluates its own batch with no data-path collective, and the job's throughput is
the points of all ranks over the slowest rank's step time.  The host logic of that
path in bench.py runs here on two gloo processes on the CPU: the max-over-ranks
reduction, the per-rank batches and the throughput formula; the reference arm does
its work on rank 0 only."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        import bench
        from paper_2603_13196_gb300 import inputs as I
        ws, r, _ = bench.dist_env()
        vals = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 0.25 * (rank + 1)])
        batch = I.workload(3).params(P=8, extra=r)          # as bench.py draws each replica's batch
        q.put((rank, ws, vals, batch))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, ws, vals, batch = q.get(timeout=120)
        out[rank] = (ws, vals, batch)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2
    # every rank sees the element-wise maximum (the slowest replica)
    assert out[0][1] == out[1][1] == [2.0, 5.0, 0.5]
    # the replicas evaluate different batches of the same workload
    assert not np.array_equal(out[0][2], out[1][2])
    assert out[0][2].shape == out[1][2].shape


def test_throughput_formula_and_single_process():
    import bench
    assert bench.replica_throughput(16384, 2, 0.2) == pytest.approx(16384 * 2 / 0.2e-3)
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]          # no process group: unchanged


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(bench.parse()) is None
    assert capsys.readouterr().out == ""
