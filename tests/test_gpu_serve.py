"""Serving (gp_server_*): partition requests that arrive over time.

Each request must come back with the blocks and cut of a gp_partition_host
call with the same arguments, whether it ran alone or overlapped with other
requests; requests larger than the device-memory budget are refused, and a
budget that admits one request at a time still serves everything.
"""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch
    import paper_2504_17615_gb300 as gpmod
    from paper_2504_17615_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return gpmod


@pytest.fixture(scope="module")
def ctx(gp):
    c = gp.Context(0)
    yield c
    c.close()


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(500), np.log(60000))))
        kind = i % 3
        if kind == 0:
            g = gg.er(n, n * int(rng.integers(4, 17)), int(rng.integers(1, 1000)))
        elif kind == 1:
            s = max(2, int(np.sqrt(n)))
            g = gg.grid2d(s, s)
        else:
            g = gg.rmat(max(9, int(np.log2(n))), 8, seed=int(rng.integers(1, 1000)))
        out.append((g, int(2 ** rng.integers(1, 8)), 0.03, int(rng.integers(1, 1 << 30))))
    return out


def _est(g):
    """The server's admission estimate (gp_response.estimate_bytes)."""
    return 4 * (4 * (g.n + 1) + 8 * g.m2 + 4 * g.n) + 8 * g.m2 + 128 * g.n + (80 << 20)


def _alone(ctx, g, k, eps, seed):
    blocks, cut, _ = ctx.gp_partition_host(g.n, g.m2, np.ascontiguousarray(g.xadj, dtype=np.int32),
                                           g.adjncy, g.vwgt, g.adjwgt, k, eps, seed)
    return blocks[:g.n].copy(), cut


def test_results_equal_alone_and_in_the_mix(gp, ctx):
    reqs = _requests(24, 3)
    ref = [_alone(ctx, *r) for r in reqs]
    srv = gp.Server(0, workers=6)
    try:
        # all at once, then a second wave submitted from another thread while the first is served
        tickets = [srv.submit(*r) for r in reqs[:16]]
        late = []
        th = threading.Thread(target=lambda: late.extend(srv.submit(*r) for r in reqs[16:]))
        th.start()
        th.join()
        served = []
        for i, t in enumerate(tickets + late):
            blocks, cut, resp = srv.wait(t)
            assert resp.status == gp.GP_OK
            assert cut == ref[i][1] and np.array_equal(blocks, ref[i][0]), f"request {i}"
            assert resp.total_ms >= resp.run_ms >= 0.0
            served.append((blocks.copy(), cut))
        # the smallest requests, served in the mix, against the CPU oracle
        small = sorted(range(len(reqs)), key=lambda i: reqs[i][0].m)[:4]
        for i in small:
            g, k, eps, seed = reqs[i]
            r = orc.partition(g, k, eps, seed)
            assert r.rc == orc.OK
            assert served[i][1] == r.cut and np.array_equal(served[i][0], r.blocks), f"request {i} vs oracle"
    finally:
        srv.close()


def test_requests_over_the_budget_are_refused(gp, ctx):
    srv = gp.Server(0, workers=2, hbm_budget=120 << 20)
    try:
        big = gg.er(300000, 3000000, 1)
        with pytest.raises(gp.GpError) as e:
            srv.submit(big, 4, 0.03, 1)
        assert e.value.status == gp.GP_ERR_BUDGET
        small = _requests(3, 5)
        small = [r for r in small if r[0].n < 2000] or [(gg.er(1000, 4000, 2), 4, 0.03, 1)]
        for r in small:
            blocks, cut, resp = srv.wait(srv.submit(*r))
            assert resp.status == gp.GP_OK and cut == _alone(ctx, *r)[1]
    finally:
        srv.close()


def test_a_one_at_a_time_budget_serves_everything(gp, ctx):
    reqs = _requests(8, 9)
    est = _est
    budget = max(est(r[0]) for r in reqs) + (1 << 20)  # any two requests together exceed it
    srv = gp.Server(0, workers=4, hbm_budget=budget)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        t0 = time.time()
        for r, t in zip(reqs, tickets):
            blocks, cut, resp = srv.wait(t)
            b1, c1 = _alone(ctx, *r)
            assert resp.status == gp.GP_OK and cut == c1 and np.array_equal(blocks, b1)
        assert time.time() - t0 < 120
    finally:
        srv.close()


def test_peak_memory_stays_within_the_admission_estimate(gp, ctx):
    """Every request's measured peak (its worker's pool, emptied before the request) is at
    most the estimate it was admitted with -- across the generator mix, including
    Erdos-Renyi requests whose levels are sparsified (Alg. 1)."""
    reqs = _requests(9, 11) + [(gg.er(200000, 1600000, 4), 8, 0.03, 5), (gg.er(60000, 600000, 6), 32, 0.03, 7)]
    for g, k, eps, seed in reqs[-2:]:
        _, _, st = ctx.gp_partition(gp.DeviceGraph.from_host(g), k, eps, seed)
        assert any(st.lv[i].triggered for i in range(st.levels))
    srv = gp.Server(0, workers=3)
    try:
        tickets = [srv.submit(*r) for r in reqs]
        for r, t in zip(reqs, tickets):
            _, _, resp = srv.wait(t)
            assert resp.status == gp.GP_OK
            assert resp.estimate_bytes == _est(r[0])
            assert 0 < resp.peak_used_bytes <= resp.peak_reserved_bytes <= resp.estimate_bytes, \
                (r[0].n, r[0].m2, resp.peak_used_bytes, resp.peak_reserved_bytes, resp.estimate_bytes)
    finally:
        srv.close()


def test_oldest_request_waits_for_at_most_max_bypass_younger_ones(gp, ctx):
    """A large request at the head of the queue that fits only alone is passed over by at
    most max_bypass younger requests, however many keep arriving."""
    big = (gg.er(200000, 1600000, 8), 16, 0.03, 3)
    smalls = [(gg.er(20000, 160000, 100 + i), 8, 0.03, i + 1) for i in range(14)]
    budget = _est(big[0]) + _est(smalls[0][0]) // 2  # the big one fits only when nothing else runs
    assert 2 * _est(smalls[0][0]) <= budget
    srv = gp.Server(0, workers=2, hbm_budget=budget)
    srv.set_max_bypass(3)
    try:
        first = srv.submit(*smalls[0])
        tb = srv.submit(*big)
        rest = [srv.submit(*r) for r in smalls[1:]]
        orders = {}
        for t in [first, tb] + rest:
            _, _, resp = srv.wait(t)
            assert resp.status == gp.GP_OK
            orders[t] = resp.start_order
        younger_first = sum(1 for t in rest if orders[t] < orders[tb])
        assert younger_first <= 3, (younger_first, orders)
    finally:
        srv.close()
