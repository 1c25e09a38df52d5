"""Batched partitioning (gp_partition_batch): many independent graphs at once.

Every item runs the same partition as a gp_partition call, so the batch must
return, item by item, exactly the blocks and cut of the single calls (and,
on small items, of the oracle), whatever the number of workers and the order
in which the workers take the items.
"""
from __future__ import annotations

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


def _mix(count, seed):
    """Mixed shapes and sizes: ER of degree 8..32, 2D and 3D grids, R-MAT; k powers of two."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(300), np.log(30000))))
        kind = i % 4
        if kind == 0:
            g = gg.er(n, n * int(rng.integers(4, 17)), int(rng.integers(1, 1000)))
        elif kind == 1:
            s = max(2, int(np.sqrt(n)))
            g = gg.grid2d(s, s)
        elif kind == 2:
            s = max(2, int(round(n ** (1 / 3))))
            g = gg.grid3d(s, s, s)
        else:
            g = gg.rmat(max(8, int(np.log2(n))), 8, seed=int(rng.integers(1, 1000)))
        if i % 5 == 0:
            g = gg.with_edge_weights(g, 7, seed=i)
        k = int(2 ** rng.integers(1, 7))
        out.append((g, k, 0.03, int(rng.integers(1, 1 << 30))))
    return out


@pytest.mark.parametrize("workers", [1, 3, 8])
def test_batch_equals_single_calls(gp, ctx, workers):
    jobs = _mix(24, workers)
    dgs = [(gp.DeviceGraph.from_host(g), k, eps, seed) for g, k, eps, seed in jobs]
    res = ctx.gp_partition_batch(dgs, workers=workers)
    for (dg, k, eps, seed), (blocks, cut) in zip(dgs, res):
        b1, c1, _ = ctx.gp_partition(dg, k, eps, seed)
        assert cut == c1
        assert np.array_equal(blocks.cpu().numpy(), b1.cpu().numpy())


def test_batch_matches_oracle_on_small_items(gp, ctx):
    jobs = [j for j in _mix(12, 7) if j[0].n <= 3000][:5]
    assert jobs
    res = ctx.gp_partition_batch([(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs], workers=4)
    for (g, k, eps, seed), (blocks, cut) in zip(jobs, res):
        r = orc.partition(g, k, eps, seed)
        assert r.rc == orc.OK and cut == r.cut
        assert np.array_equal(blocks.cpu().numpy(), r.blocks)


def test_batch_reports_a_failing_item_and_finishes_the_others(gp, ctx):
    jobs = _mix(6, 11)
    dgs = [(gp.DeviceGraph.from_host(g), k, eps, seed) for g, k, eps, seed in jobs]
    dgs[2] = (dgs[2][0], 0, 0.03, 1)  # k = 0 is invalid
    res = ctx.gp_partition_batch(dgs, workers=3, check=False)
    assert res[2][2] == gp.GP_ERR_INVALID
    for i, (dg, k, eps, seed) in enumerate(dgs):
        if i == 2:
            continue
        assert res[i][2] == gp.GP_OK
        _, c1, _ = ctx.gp_partition(dg, k, eps, seed)
        assert res[i][1] == c1
