"""Full-size checks on the workloads the benchmark times, through the C-ABI.

The oracle cannot run a whole partition of the 2^26-node Erdos-Renyi graph
in test time, so at full size the GPU path is checked by

* bit-exact parity with the oracle on what the oracle can compute there: the
  first LP sub-round of level 1 (every active node's rating, choice,
  acceptance and move over 1/8 of the 1.34e9 entries);
* exact recomputation on the host of sampled outputs: contracted rows of
  sampled coarse nodes, the sparsifier's keep decision on every entry of
  sampled rows;
* properties that hold at any size: node weight preserved, coarse edge
  weight equal to the inter-cluster weight (Sec. 2), the threshold's
  selection definition and the kept count within the binomial slack
  (Sec. 4.2), the per-level rules of Alg. 1 (m_hat, trigger, shrink stop),
  balance under L_max and the reported cut equal to the cut recomputed
  from the blocks.

Everything runs in the launch configuration of ``bench.py`` (the same
gp_partition call, k = 128, eps = 0.03, seed 1, default configuration).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu

C3 = dict(n=1 << 26, m=671_088_640, k=128, eps=0.03, seed=1)
C2 = dict(scale=24, ef=16, k=64, eps=0.03, seed=1)
SAMPLES = 2000


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


@pytest.fixture(scope="module")
def c3(gp):
    g = gg.er(C3["n"], C3["m"], C3["seed"])
    return g, gp.DeviceGraph.from_host(g)


def host_cut(g, blk):
    """cut = 1/2 sum over CSR entries whose endpoints lie in different blocks, in row chunks."""
    xadj = np.asarray(g.xadj, dtype=np.int64)
    total = 0
    step = 1 << 22
    for r0 in range(0, g.n, step):
        r1 = min(g.n, r0 + step)
        e0, e1 = int(xadj[r0]), int(xadj[r1])
        rows = np.repeat(np.arange(r0, r1, dtype=np.int64), np.diff(xadj[r0:r1 + 1]))
        diff = blk[rows] != blk[g.adjncy[e0:e1]]
        total += int(np.asarray(g.adjwgt[e0:e1], dtype=np.int64)[diff].sum())
    return total // 2


def inter_cluster_weight(g, cmap):
    xadj = np.asarray(g.xadj, dtype=np.int64)
    total = 0
    step = 1 << 22
    for r0 in range(0, g.n, step):
        r1 = min(g.n, r0 + step)
        e0, e1 = int(xadj[r0]), int(xadj[r1])
        rows = np.repeat(np.arange(r0, r1, dtype=np.int64), np.diff(xadj[r0:r1 + 1]))
        diff = cmap[rows] != cmap[g.adjncy[e0:e1]]
        total += int(np.asarray(g.adjwgt[e0:e1], dtype=np.int64)[diff].sum())
    return total


def check_levels(st, cfg_o):
    """Alg. 1 per level: m_hat, the trigger, the kept count, the shrink stop rule."""
    for i in range(st.levels):
        L = st.lv[i]
        assert L.m_coarse <= L.m
        assert L.m_hat == orc.m_hat(L.m, L.n, L.n_next, cfg_o)
        assert bool(L.triggered) == orc.trigger(L.m_coarse, L.m_hat, cfg_o)
        if L.triggered:
            assert abs(L.m_next - L.m_hat) <= 6 * math.sqrt(L.m_hat) + 1
        else:
            assert L.m_next == L.m_coarse
        assert 21 * L.n_next <= 20 * L.n  # levels that shrink less are discarded (R13)
        if i + 1 < st.levels:
            assert st.lv[i + 1].n == L.n_next and st.lv[i + 1].m == L.m_next


def test_c3_partition_properties(gp, ctx, c3):
    g, dg = c3
    k, eps, seed = C3["k"], C3["eps"], C3["seed"]
    blocks, cut, st = ctx.gp_partition(dg, k, eps, seed)
    blk = blocks.cpu().numpy()
    W = int(g.n)
    assert st.W == W
    assert st.U == orc.cluster_bound(W, k)
    assert st.Lmax == orc.lmax(W, k, orc.eps_to_ppm(eps))
    assert blk.min() >= 0 and blk.max() < k
    assert np.bincount(blk, minlength=k).max() <= st.Lmax
    assert cut == host_cut(g, blk)
    check_levels(st, orc.Config.default())
    assert any(st.lv[i].triggered for i in range(st.levels))  # the low-modularity case sparsifies


def test_c3_first_subround_matches_oracle(gp, ctx, c3):
    g, dg = c3
    U = orc.cluster_bound(g.n, C3["k"])
    kw = dict(dbg_max_subrounds=1, two_hop=0, isolated=0)
    _, nc, st, label = ctx.gp_coarsen(dg, U, 1, C3["seed"], gp.default_config(**kw), want_label=True)
    olabel, oncl, ost = orc.cluster(g, U, 1, C3["seed"], orc.Config.default(**kw))
    assert np.array_equal(label.cpu().numpy(), olabel)
    assert (nc, st.lp_subrounds, st.lp_moves) == (oncl, ost.lp_subrounds, ost.lp_moves)


@pytest.fixture(scope="module")
def c3_level1(gp, ctx, c3):
    g, dg = c3
    U = orc.cluster_bound(g.n, C3["k"])
    cmap_d, nc, st = ctx.gp_coarsen(dg, U, 1, C3["seed"])
    cmap = cmap_d.cpu().numpy()
    cg = ctx.gp_contract(dg, cmap_d, nc)
    return U, cmap, nc, st, cg, cg.to_host()


def test_c3_level1_clustering_properties(gp, ctx, c3, c3_level1):
    g, _ = c3
    U, cmap, nc, st, _, _ = c3_level1
    assert cmap.min() == 0 and cmap.max() == nc - 1
    sizes = np.bincount(cmap, minlength=nc)
    assert sizes.min() >= 1  # dense ids (R11)
    assert sizes.max() <= U  # unit weights: cluster weight = size <= U
    assert st.clusters_final == nc and st.n_next == nc
    assert st.clusters_final <= st.clusters_2hop <= st.clusters_lp < g.n


def test_c3_level1_modularity(gp, ctx, c3, c3_level1):
    """Sec. 5 on the level-1 clustering: exact totals against the host, and Lemma 2's bound
    below the weight fraction the contraction keeps."""
    import torch
    g, dg = c3
    U, cmap, nc, st, cg, h = c3_level1
    M = ctx.gp_modularity(dg, torch.from_numpy(cmap).cuda(), nc)
    inter = inter_cluster_weight(g, cmap)
    assert M.w_total == g.m2 and M.w_internal == g.m2 - inter
    vol = np.bincount(cmap, weights=np.diff(np.asarray(g.xadj, dtype=np.int64)), minlength=nc).astype(np.int64)
    assert M.vol_max == int(vol.max())
    assert M.vol_sq == int((vol * vol).sum())
    assert M.q <= M.inside <= M.q + M.alpha  # Lemma 2
    assert int(np.asarray(h.adjwgt, dtype=np.int64).sum()) / g.m2 >= M.bound


def test_c3_level1_contraction_sampled(gp, ctx, c3, c3_level1):
    g, _ = c3
    U, cmap, nc, st, cg, h = c3_level1
    assert h.n == nc
    # node weights: sum over members (unit fine weights)
    assert np.array_equal(np.asarray(h.vwgt, dtype=np.int64), np.bincount(cmap, minlength=nc))
    # edge weight: the coarse graph carries exactly the inter-cluster weight, both directions
    assert int(np.asarray(h.adjwgt, dtype=np.int64).sum()) == inter_cluster_weight(g, cmap)
    hx = np.asarray(h.xadj, dtype=np.int64)
    # sampled coarse nodes: rows recomputed from the fine graph
    order = np.argsort(cmap, kind="stable")
    starts = np.concatenate([[0], np.cumsum(np.bincount(cmap, minlength=nc))])
    rng = np.random.default_rng(5)
    gx = np.asarray(g.xadj, dtype=np.int64)
    for A in rng.integers(0, nc, SAMPLES):
        members = order[starts[A]:starts[A + 1]]
        nb = np.concatenate([g.adjncy[gx[v]:gx[v + 1]] for v in members])
        wb = np.concatenate([g.adjwgt[gx[v]:gx[v + 1]] for v in members]).astype(np.int64)
        cb = cmap[nb]
        keep = cb != A
        keys, inv = np.unique(cb[keep], return_inverse=True)
        wsum = np.bincount(inv, weights=wb[keep]).astype(np.int64) if len(keys) else np.zeros(0, np.int64)
        row = np.asarray(h.adjncy[hx[A]:hx[A + 1]], dtype=np.int64)
        roww = np.asarray(h.adjwgt[hx[A]:hx[A + 1]], dtype=np.int64)
        o = np.argsort(row)
        assert np.array_equal(row[o], keys), f"coarse row {A}"
        assert np.array_equal(roww[o], wsum), f"coarse weights {A}"


def test_c3_level1_sparsify_sampled(gp, ctx, c3, c3_level1):
    g, _ = c3
    U, cmap, nc, st, cg, h = c3_level1
    m = g.m2 // 2
    m_coarse = cg.m2 // 2
    cfg = orc.Config.default()
    mh = orc.m_hat(m, g.n, nc, cfg)
    assert orc.trigger(m_coarse, mh, cfg)  # the ER level-1 case of Alg. 1
    sg, sst = ctx.gp_sparsify(cg, mh, 2, C3["seed"])
    s = sg.to_host()
    w = np.asarray(h.adjwgt, dtype=np.int64)
    wt = sst.omega_t
    n_gt = int((w > wt).sum()) // 2
    n_eq = int((w == wt).sum()) // 2
    # the selection definition of omega_t (Sec. 4.2)
    assert (sst.n_greater, sst.n_equal) == (n_gt, n_eq)
    assert n_gt < mh <= n_gt + n_eq
    assert sst.threshold == ((mh - n_gt) << 32) // n_eq
    assert abs(sg.m2 // 2 - mh) <= 6 * math.sqrt(mh) + 1
    # sampled rows: every entry's keep decision recomputed, kept entries in row order
    key = orc.key(C3["seed"], orc.TAG_SPARSE, 2, 0)
    hx = np.asarray(h.xadj, dtype=np.int64)
    sx = np.asarray(s.xadj, dtype=np.int64)
    rng = np.random.default_rng(9)
    for A in rng.integers(0, nc, SAMPLES):
        row = h.adjncy[hx[A]:hx[A + 1]]
        roww = h.adjwgt[hx[A]:hx[A + 1]]
        kept = []
        for B, x in zip(row.tolist(), roww.tolist()):
            lo, hi = (A, B) if A < B else (B, A)
            if x > wt or (x == wt and orc.h32(key, lo, hi) < sst.threshold):
                kept.append((B, x))
        got = list(zip(s.adjncy[sx[A]:sx[A + 1]].tolist(), s.adjwgt[sx[A]:sx[A + 1]].tolist()))
        assert got == kept, f"row {A}"


def test_c2_rmat_partition_properties(gp, ctx):
    g = gg.rmat(C2["scale"], C2["ef"], seed=C2["seed"])
    dg = gp.DeviceGraph.from_host(g)
    k, eps = C2["k"], C2["eps"]
    blocks, cut, st = ctx.gp_partition(dg, k, eps, C2["seed"])
    blk = blocks.cpu().numpy()
    assert st.Lmax == orc.lmax(g.n, k, orc.eps_to_ppm(eps))
    assert np.bincount(blk, minlength=k).max() <= st.Lmax
    assert cut == host_cut(g, blk)
    check_levels(st, orc.Config.default())
    # first LP sub-round of level 1 bit-exact against the oracle (skewed degrees: every rating kernel)
    U = orc.cluster_bound(g.n, k)
    kw = dict(dbg_max_subrounds=1, two_hop=0, isolated=0)
    _, nc, st1, label = ctx.gp_coarsen(dg, U, 1, C2["seed"], gp.default_config(**kw), want_label=True)
    olabel, oncl, _ = orc.cluster(g, U, 1, C2["seed"], orc.Config.default(**kw))
    assert np.array_equal(label.cpu().numpy(), olabel) and nc == oncl
