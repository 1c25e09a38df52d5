"""The batched engine of gp_partition_batch: one persistent launch whose CTAs
take whole graphs from a device-side queue and partition each inside the CTA.

It runs the same method and readings as the per-graph path, so every item
must equal the oracle bit for bit -- blocks, cut and every per-level record of
Alg. 1 -- and equal a gp_partition call with the same arguments, for every
CTA size, on every graph shape (hubs above the warp and the CTA table sizes,
isolated nodes, weights), under configuration variants, and when an item
falls back to the per-graph path (arena too small, exact-count sparsifier).
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from _util import hand, isolated, matching, star

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


def _engine_on(ctx, threads=512, **kw):
    ctx.batch_set_tuning(engine=1, threads=threads, max_entries=1 << 26, max_nodes=1 << 24, **kw)


def _star_plus(leaves, extra, seed):
    """A hub of `leaves` neighbours plus a random graph on the leaves (hub rows above 2048 entries)."""
    rng = np.random.default_rng(seed)
    e = [(0, i) for i in range(1, leaves + 1)]
    for _ in range(extra):
        a, b = rng.integers(1, leaves + 1, 2)
        if a != b:
            e.append((int(min(a, b)), int(max(a, b))))
    e = sorted(set(e))
    return hand(leaves + 1, e, name=f"starplus{leaves}")


def _oracle_jobs():
    jobs = []
    jobs.append((gg.er(3000, 12000, 5), 2, 0.03, 11))
    jobs.append((gg.er(5000, 40000, 6), 8, 0.03, 12))
    jobs.append((gg.with_edge_weights(gg.er(4000, 20000, 7), 9, seed=3), 4, 0.05, 13))
    jobs.append((gg.grid2d(60, 50), 3, 0.03, 14))
    jobs.append((gg.grid3d(14, 14, 14), 16, 0.03, 15))
    jobs.append((gg.rmat(12, 8, seed=4), 8, 0.03, 16))
    jobs.append((star(600), 2, 0.03, 17))
    jobs.append((_star_plus(3000, 6000, 1), 4, 0.03, 18))
    jobs.append((isolated(700), 5, 0.03, 19))
    jobs.append((matching(900), 4, 0.03, 20))
    jobs.append((gg.with_isolated(gg.er(2000, 6000, 8), 500), 6, 0.03, 21))
    jobs.append((gg.er(65536, 524288, 1), 2, 0.03, 1))  # the C1 configuration (sparsification triggers)
    jobs.append((gg.with_node_weights(gg.er(2500, 10000, 9), 5), 7, 0.03, 22))
    jobs.append((gg.rmat(10, 16, seed=2), 64, 0.03, 23))
    return jobs


def _check_against_oracle(res, jobs, cfg_kw=None):
    for (g, k, eps, seed), (blocks, cut, eng, st) in zip(jobs, res):
        r = orc.partition(g, k, eps, seed, orc.Config.default(**(cfg_kw or {})))
        assert r.rc == orc.OK
        assert cut == r.cut, g.name
        assert np.array_equal(blocks.cpu().numpy(), r.blocks), g.name
        assert st.levels == r.stats.levels, g.name
        for i in range(st.levels):
            a, b = st.lv[i], r.stats.lv[i]
            for f in ("n", "n_next", "m", "m_coarse", "m_hat", "m_next", "triggered", "omega_t", "n_greater",
                      "n_equal", "threshold", "lp_subrounds", "lp_moves", "clusters_lp", "clusters_2hop",
                      "clusters_final"):
                assert getattr(a, f) == getattr(b, f), (g.name, i, f)
        assert (st.U, st.Lmax, st.W, st.ip_cut, st.rebalance_moves, st.n_coarsest, st.cut) == \
            (r.stats.U, r.stats.Lmax, r.stats.W, r.stats.ip_cut, r.stats.rebalance_moves, r.stats.n_coarsest,
             r.cut), g.name


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_engine_matches_oracle(gp, ctx, threads):
    jobs = _oracle_jobs()
    _engine_on(ctx, threads)
    dgs = [(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs]
    res = ctx.gp_partition_batch(dgs, workers=2, details=True)
    assert all(r[2] == 1 for r in res), "every item ran on the engine"
    _check_against_oracle(res, jobs)


def _mix(count, seed, nmax=30000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(300), np.log(nmax))))
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


def test_engine_equals_single_calls_on_a_mix(gp, ctx):
    jobs = _mix(40, 3, nmax=100000)
    dgs = [(gp.DeviceGraph.from_host(g), k, eps, seed) for g, k, eps, seed in jobs]
    _engine_on(ctx, 512)
    res = ctx.gp_partition_batch(dgs, workers=4, details=True)
    assert all(r[2] == 1 for r in res)
    for (dg, k, eps, seed), (blocks, cut, eng, st) in zip(dgs, res):
        b1, c1, s1 = ctx.gp_partition(dg, k, eps, seed)
        assert cut == c1
        assert np.array_equal(blocks.cpu().numpy(), b1.cpu().numpy())
        assert st.levels == s1.levels and st.ip_cut == s1.ip_cut


@pytest.mark.parametrize("kw", [{"sparsifier": 0}, {"sparsifier": 2}, {"ref_rounds": 0}, {"coarsest_factor": 20},
                                {"ip_trials": 3}, {"lp_subrounds": 3}, {"two_hop": 0, "isolated": 0},
                                {"dbg_max_subrounds": 5}, {"lp_rounds": 1, "ref_rounds": 2}])
def test_engine_config_variants(gp, ctx, kw):
    jobs = [(gg.er(6000, 30000, 3), 4, 0.05, 4), (gg.with_isolated(gg.rmat(11, 8, seed=5), 300), 8, 0.03, 5),
            (star(2500), 3, 0.03, 6)]
    _engine_on(ctx, 256)
    dgs = [(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs]
    res = ctx.gp_partition_batch(dgs, workers=2, cfg=gp.default_config(**kw), details=True)
    assert all(r[2] == 1 for r in res)
    _check_against_oracle(res, jobs, kw)


def test_engine_leaves_the_exact_sparsifier_to_the_per_graph_path(gp, ctx):
    jobs = [(gg.er(5000, 40000, 6), 8, 0.03, 12)]
    _engine_on(ctx, 512)
    dgs = [(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs]
    res = ctx.gp_partition_batch(dgs, workers=1, cfg=gp.default_config(sparsifier=3), details=True)
    assert res[0][2] == 0
    _check_against_oracle(res, jobs, {"sparsifier": 3})


def test_engine_small_arena_hands_items_to_the_per_graph_path(gp, ctx):
    jobs = [(gg.er(20000, 100000, 2), 4, 0.03, 3), (gg.grid2d(20, 20), 2, 0.03, 4)]
    _engine_on(ctx, 512, arena_bytes=1 << 18)
    dgs = [(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs]
    res = ctx.gp_partition_batch(dgs, workers=2, details=True)
    assert res[0][2] == 0, "the large item outgrew its arena and ran on the per-graph path"
    assert res[1][2] == 1, "the small one fits"
    _check_against_oracle(res, jobs)


def test_engine_trivial_items(gp, ctx):
    jobs = [(gg.er(500, 2000, 1), 1, 0.03, 1), (isolated(1), 2, 0.03, 1), (isolated(2), 2, 0.03, 1),
            (gg.grid2d(3, 3), 2, 0.03, 1), (gg.er(200, 600, 2), 4, 0.5, 7)]
    _engine_on(ctx, 1024)
    dgs = [(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs]
    res = ctx.gp_partition_batch(dgs, workers=1, details=True)
    assert all(r[2] == 1 for r in res)
    _check_against_oracle(res, jobs)


def test_engine_reports_invalid_items_like_gp_partition(gp, ctx):
    good = gg.er(1000, 4000, 1)
    loop = hand(4, [(0, 1), (1, 2), (2, 3)])
    loop.adjncy = loop.adjncy.copy()
    loop.adjncy[0] = 0  # node 0 lists itself
    asym = hand(4, [(0, 1), (1, 2), (2, 3)], weights=[1, 2, 3])
    asym.adjwgt = asym.adjwgt.copy()
    asym.adjwgt[0] = 5  # w(0,1) != w(1,0)
    heavy = hand(4, [(0, 1), (1, 2), (2, 3)], vwgt=[100, 1, 1, 1])
    jobs = [(good, 2, 0.03, 1), (loop, 2, 0.03, 1), (asym, 2, 0.03, 1), (heavy, 2, 0.03, 1), (good, 0, 0.03, 1)]
    _engine_on(ctx, 512)
    dgs = [(gp.DeviceGraph.from_host(g), k, e, s) for g, k, e, s in jobs]
    res = ctx.gp_partition_batch(dgs, workers=1, check=False, details=True)
    expect = [gp.GP_OK, gp.GP_ERR_INVALID, gp.GP_ERR_INVALID, gp.GP_ERR_INFEASIBLE, gp.GP_ERR_INVALID]
    assert [r[2] for r in res] == expect
    for (dg, k, e, s), r in zip(dgs, res):
        try:
            _, c1, _ = ctx.gp_partition(dg, k, e, s)
            st1 = gp.GP_OK
        except gp.GpError as err:
            st1 = err.status
        assert st1 == r[2]
    r0 = orc.partition(good, 2, 0.03, 1)
    assert res[0][1] == r0.cut and np.array_equal(res[0][0].cpu().numpy(), r0.blocks)


def test_autotune_installs_a_table_and_results_stay_identical(gp, ctx):
    jobs = _mix(24, 9, nmax=60000)
    dgs = [(gp.DeviceGraph.from_host(g), k, eps, seed) for g, k, eps, seed in jobs]
    t = ctx.batch_autotune(dgs, workers=4)
    d = t.as_dict()
    assert t.threads in (256, 512, 1024) and t.classes >= 1 and d["class_table"]
    assert ctx.batch_tuning().threads == t.threads
    res = ctx.gp_partition_batch(dgs, workers=4, details=True)
    for (dg, k, eps, seed), (blocks, cut, eng, st) in zip(dgs, res):
        if eng:
            assert dg.m2 <= t.max_entries
        b1, c1, _ = ctx.gp_partition(dg, k, eps, seed)
        assert cut == c1 and np.array_equal(blocks.cpu().numpy(), b1.cpu().numpy())
    ctx.batch_set_tuning()  # defaults again


def test_engine_beside_the_per_graph_path(gp, ctx):
    """Small items on the engine while the larger ones run on the per-graph path at the same time."""
    jobs = _mix(48, 5, nmax=60000)
    dgs = [(gp.DeviceGraph.from_host(g), k, eps, seed) for g, k, eps, seed in jobs]
    ctx.batch_set_tuning(engine=1, threads=512, max_entries=1 << 15, max_nodes=1 << 24)
    res = ctx.gp_partition_batch(dgs, workers=4, details=True)
    flags = [r[2] for r in res]
    assert 0 < sum(flags) < len(flags), "both paths ran"
    for (dg, k, eps, seed), (blocks, cut, eng, st) in zip(dgs, res):
        assert eng == (1 if dg.m2 <= 1 << 15 else 0)
        b1, c1, _ = ctx.gp_partition(dg, k, eps, seed)
        assert cut == c1 and np.array_equal(blocks.cpu().numpy(), b1.cpu().numpy())
    ctx.batch_set_tuning()
