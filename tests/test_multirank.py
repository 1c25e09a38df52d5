"""The benchmark's multi-rank path on CPU: two gloo ranks, as torchrun starts them.

With N > 1 every rank partitions its own replica of the workload graph (the
method does not shard one graph), so the host logic to cover is: rank 0 draws
the graph and the others read the same CSR from a shared file, and the timing
is the maximum over ranks.
"""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = dict(name="er_test", n=5000, m=40000, k=4, eps=0.03, seed=3)
        g = bench.make_graph(w, rank, world)
        digest = int(np.asarray(g.xadj, dtype=np.int64).sum() * 31 + np.asarray(g.adjncy, dtype=np.int64).sum())
        got = bench.max_over_ranks([rank + 1.0, 10.0 - rank, digest])
        out.put((rank, g.n, g.m2, digest, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_graph_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, m0, d0, got0), (r1, n1, m1, d1, got1) = res
    assert (n0, m0, d0) == (n1, m1, d1)            # the same replica on both ranks
    assert got0 == got1 == [2.0, 10.0, float(d0)]  # maximum over ranks
