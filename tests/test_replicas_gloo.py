"""The N > 1 path of bench.py without a GPU: two gloo ranks on CPU.

The apply does not shard.  With N GPUs, bench.py runs N independent replicas, each applying its
own batch, and reports the whole job's throughput over the slowest rank's time. These tests check
that host logic on two CPU processes:
- the barrier;
- the max over ranks;
- the per-rank input seeds, which must differ;
- the reference arm, which only rank 0 runs.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import workloads as W
    got_ws, got_rank, _ = bench.dist_init()
    assert (got_ws, got_rank) == (ws, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(ws)
    slowest = bench.max_over_ranks(ws, 1.0 + rank)       # rank r "took" 1 + r seconds
    # each replica draws its own batch (the seeding bench.py uses for ranks > 1)
    f = W.complex_gaussian((4, 4, 2), 10_000 + rank)
    g = torch.zeros(2, 4, 4, 2, dtype=torch.complex128)
    g[rank] = f
    dist.all_reduce(g)
    q.put((rank, slowest, bool(torch.equal(g[0], g[1]))))
    dist.destroy_process_group()


def test_two_replicas_share_the_slowest_time_and_draw_different_batches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r for r, _, _ in res] == [0, 1]
    assert all(slowest == 2.0 for _, slowest, _ in res)      # max over ranks, seen by every rank
    assert not res[0][2]                                       # the two batches differ


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    args = bench.parse()
    bench.reference_arm(args, 2, 1)        # rank 1 of 2: no work, no output
    assert capsys.readouterr().out == ""
