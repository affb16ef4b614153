"""Host logic of the benchmark's multi-rank launch on CPU (gloo, world size 2): each rank runs an
independent replica, the step time reported is the slowest rank's, and the reference arm runs on
rank 0 only (the other ranks exit without work)."""

import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w = bench._dist()
    # rank r reports (r + 1) * 10 ms; every rank must see the slowest one
    got = bench.max_over_ranks(dist, (r + 1) * 10.0)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, got))


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 20.0), (1, 2, 20.0)]


def test_single_rank_needs_no_process_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    sys.path.insert(0, ROOT)
    import bench
    dist, rank, ws = bench._dist()
    assert dist is None and (rank, ws) == (0, 1)
    assert bench.max_over_ranks(dist, 3.5) == 3.5


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    sys.path.insert(0, ROOT)
    import bench
    args = bench.argparse.Namespace(workload=bench.WORKLOAD, steps=1, warmup=0, cpu_budget=1.0)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
