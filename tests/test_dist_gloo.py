"""The benchmark's multi-rank logic (replicas, weak scaling): rank
environment, barrier, slowest-rank time and summed work, run as two gloo
ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    r, local, w = bench.dist_env()
    d = bench.init_dist(w, "gloo")
    bench.barrier(d)
    slowest = bench.max_over_ranks(d, 1.0 + rank)          # per-step ms of each rank
    total = bench.sum_over_ranks(d, 1000.0 * (rank + 1))    # nodes advanced by each rank
    out.put((r, local, w, slowest, total))
    d.destroy_process_group()


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
    assert [r[0] for r in res] == [0, 1] and all(r[2] == 2 for r in res)
    assert all(r[3] == 2.0 for r in res)        # max over ranks
    assert all(r[4] == 3000.0 for r in res)     # sum over ranks


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 0, 1)
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 2.5) == 2.5 and bench.sum_over_ranks(None, 7.0) == 7.0
