"""Host logic of the N > 1 bench launch (replicas, one process per GPU) on
CPU with gloo, world size 2: distinct seeds per rank, barrier on both sides of
the timed region, maximum over ranks."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_env()
        dev = torch.device("cpu")
        bench.sync_all(w, dev)
        mx = bench.max_over_ranks([1.0 + r, 10.0 - r], w, dev)
        bench.sync_all(w, dev)
        q.put((r, w, loc, bench.rank_seed(7, r), mx))
    finally:
        dist.destroy_process_group()


def test_two_rank_host_logic():
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
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 for r in res)
    assert res[0][3] != res[1][3]                       # every replica solves its own system
    assert all(r[4] == [2.0, 10.0] for r in res)        # max over ranks, seen by every rank


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, torch.device("cpu")) == [3.0, 4.0]
    bench.sync_all(1, torch.device("cpu"))
    assert bench.workload_config(40, "x", "f64")["n"] == 201720
