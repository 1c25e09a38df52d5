"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
test vectors, closed forms from the paper, hand-worked examples, invariants
the paper states, brute force on tiny graphs, and statistical expectations.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from tests._util import (brute_force_opt, check_csr, clique, hand, isolated, matching, path,
                         row_index, star, to_sets)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GOLD = 0x9E3779B97F4A7C15


# ------------------------------------------------------------------ hash pin

def _vectors():
    out = []
    for line in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")):
        line = line.split("#")[0].strip()
        if line:
            i, h = line.split()
            out.append((int(i), int(h, 16)))
    return out


def test_hash_finaliser_matches_published_splitmix64_vectors():
    # h32(key, x, y) = top 32 bits of mix(key ^ (x << 32 | y)); with key = 0 the
    # input is the SplitMix64 state (i + 1) * gamma, whose outputs are published.
    for i, expect in _vectors():
        state = ((i + 1) * GOLD) & ((1 << 64) - 1)
        got = orc.h32(0, state >> 32, state & 0xFFFFFFFF)
        assert got == expect >> 32, (i, hex(got), hex(expect))


def test_generator_words_match_published_splitmix64_vectors():
    # graphgen word t of stream s is fin(fin(s + SALT) + (t + 1) * gamma); the
    # seed that zeroes the inner finaliser reduces it to the plain sequence.
    salt = 0x632BE59BD9B4E019
    seed = (-salt) & ((1 << 64) - 1)
    w = gg.word(seed, np.arange(4, dtype=np.uint64))
    for i, expect in _vectors():
        assert int(w[i]) == expect


def test_hash_keys_separate_streams():
    ks = {orc.key(1, t, l, r) for t in range(1, 11) for l in range(4) for r in range(6)}
    assert len(ks) == 10 * 4 * 6
    assert orc.key(1, 1, 1, 0) != orc.key(2, 1, 1, 0)


# ------------------------------------------------------------ closed forms

def _golden_params():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_parameters.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = v
    return out


def test_default_config_is_the_papers():
    p = _golden_params()
    c = orc.Config.default()
    assert f"{c.tau_e_num}/{c.tau_e_den}" == p["tau_e"]
    assert f"{c.tau_d_num}/{c.tau_d_den}" == p["tau_d"]
    assert str(c.rho_num // c.rho_den) == p["rho"] and c.rho_num % c.rho_den == 0
    assert str(c.cluster_factor) == p["cluster_factor"]
    assert str(c.coarsest_factor) == p["coarsest_factor"]
    assert f"{c.shrink_num}/{c.shrink_den}" == p["max_shrink"]


def test_lmax_closed_form():
    # L_max = (1 + eps) ceil(c(V) / k), Sec. 2
    assert orc.lmax(65536, 2, 30000) == 33751          # 32768 * 1.03 = 33751.04
    assert orc.lmax(10, 2, 30000) == 5                 # 5 * 1.03 = 5.15
    assert orc.lmax(11, 2, 30000) == 6                 # ceil(5.5) = 6 -> 6.18
    assert orc.lmax(1 << 26, 128, 30000) == 540016     # 524288 * 1.03 = 540016.64
    for W, k, e in [(1000, 3, 30000), (999, 7, 10000), (12345, 64, 30000), (7, 8, 500000)]:
        exact = math.ceil(W / k) * (1 + e / 1e6)
        assert orc.lmax(W, k, e) == math.floor(exact + 1e-9)


def test_cluster_bound_closed_form():
    # U = c(V) / (160 k), Sec. 4.3
    assert orc.cluster_bound(65536, 2) == 204
    assert orc.cluster_bound(1 << 24, 64) == 1638
    assert orc.cluster_bound(1 << 26, 128) == 3276
    assert orc.cluster_bound(100, 64) == 1


def test_m_hat_and_trigger_closed_form():
    # m_hat = min(tau_e m, tau_d m / n * n'), trigger iff m' > rho m_hat (Alg. 1)
    cfg = orc.Config.default()
    for m, n, n2 in [(524288, 65536, 22967), (1000, 100, 40), (10, 10, 10), (7, 3, 1)]:
        expect = min(m // 2, (m * n2) // (2 * n))
        assert orc.m_hat(m, n, n2, cfg) == expect
    assert orc.trigger(401, 100, cfg) and not orc.trigger(400, 100, cfg)
    # with tau_e = tau_d = 1/2 and rho = 4: trigger iff m'/m > 2 n'/n (up to flooring)
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(10, 10**6)); n2 = int(rng.integers(1, n + 1))
        m = int(rng.integers(n, 20 * n)); mc = int(rng.integers(0, m + 1))
        mh = orc.m_hat(m, n, n2, cfg)
        assert orc.trigger(mc, mh, cfg) == (mc > 4 * mh)
        if abs(mc * n - 2 * m * n2) > 8 * n:   # away from the flooring boundary
            assert orc.trigger(mc, mh, cfg) == (mc * n > 2 * m * n2)


# ------------------------------------------------------------- validation

def test_validate_accepts_generated_graphs():
    for g in (gg.er(200, 800, 3), gg.grid2d(5, 7), gg.rmat(8, 8)):
        rc, W = orc.validate(g)
        assert rc == orc.OK and W == g.n


def test_validate_rejects_bad_inputs():
    g = path(4)
    bad = []
    b = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    b.adjwgt[0] = 5                                    # asymmetric weight
    bad.append((b, orc.INVALID))
    b = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    b.vwgt[2] = 0                                      # zero node weight
    bad.append((b, orc.INVALID))
    b = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    b.adjncy[0] = 0                                    # self-loop at node 0
    bad.append((b, orc.INVALID))
    x = np.array([0, 2, 3, 3], dtype=np.int64)         # missing reverse entry
    bad.append((gg.Graph(3, x, np.array([1, 2, 0], np.int32), np.ones(3, np.int32),
                         np.ones(3, np.int32)), orc.INVALID))
    b = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    b.adjwgt[:] = 2**30                                 # total edge weight overflows int32
    bad.append((b, orc.OVERFLOW))
    for b, rc in bad:
        assert orc.validate(b)[0] == rc
    # infeasible: a node heavier than L_max
    h = path(4)
    h.vwgt = np.array([1, 1, 1, 9], np.int32)
    assert orc.partition(h, 2, 0.03, 1).rc == orc.INFEASIBLE


# ------------------------------------------------------------- contraction

def test_contraction_hand_examples():
    # path 0-1-2-3 with clusters {0,1},{2,3}: one coarse edge of weight 1, weights 2, 2
    c = orc.contract(path(4), np.array([0, 0, 1, 1]), 2)
    assert list(c.vwgt) == [2, 2] and to_sets(c) == {(0, 1): 1, (1, 0): 1}
    # K4 as one cluster: one node of weight 4, no edges
    k4 = hand(4, clique(4))
    c = orc.contract(k4, np.zeros(4, np.int32), 1)
    assert list(c.vwgt) == [4] and c.m2 == 0
    # two triangles joined by two edges, each triangle a cluster: one edge of weight 2
    tt = hand(6, clique(3) + clique(3, 3) + [(0, 3), (1, 4)])
    c = orc.contract(tt, np.array([0, 0, 0, 1, 1, 1]), 2)
    assert list(c.vwgt) == [3, 3] and to_sets(c) == {(0, 1): 2, (1, 0): 2}
    # weighted: parallel fine edges add up
    wg = hand(4, [(0, 2), (0, 3), (1, 3), (0, 1)], weights=[5, 7, 11, 13], vwgt=[2, 3, 4, 5])
    c = orc.contract(wg, np.array([0, 0, 1, 1]), 2)
    assert list(c.vwgt) == [5, 9] and to_sets(c) == {(0, 1): 23, (1, 0): 23}


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_contraction_invariants(seed):
    g = gg.with_node_weights(gg.with_edge_weights(gg.er(500, 3000, seed), 9), 5)
    rng = np.random.default_rng(seed)
    nc = 60
    cmap = rng.integers(0, nc, g.n).astype(np.int32)
    cmap[:nc] = np.arange(nc)                           # every coarse id used
    c = orc.contract(g, cmap, nc)
    check_csr(c)
    assert c.vwgt.sum() == g.vwgt.sum()                 # node weight preserved (Sec. 2)
    rows = row_index(g)
    inter = cmap[rows] != cmap[g.adjncy]
    assert c.adjwgt.sum() == g.adjwgt[inter].sum()      # coarse weight = inter-cluster weight
    # each coarse edge weight is the weight between its two clusters
    ent = to_sets(c)
    for (A, B), w in list(ent.items())[:200]:
        sel = (cmap[rows] == A) & (cmap[g.adjncy] == B)
        assert g.adjwgt[sel].sum() == w


# -------------------------------------------------------------- clustering

def _cluster_weights(g, label):
    return np.bincount(label, weights=g.vwgt, minlength=g.n)


def test_perfect_matching_clusters_every_edge():
    # Each edge becomes one cluster, except a pair whose two ends are active in
    # the same sub-round of every round: they swap labels each time and stay
    # apart (synchronous sub-rounds, R4); 2-hop cannot join them (different
    # favourites).
    g = matching(500)
    cfg = orc.Config.default()
    for seed in (1, 2, 3):
        label, ncl, _ = orc.cluster(g, 4, 1, seed)
        keys = [orc.key(seed, orc.TAG_ACT, 1, r) for r in range(cfg.lp_rounds)]
        stuck = sum(all(orc.h32(k, 2 * i, 0) % 8 == orc.h32(k, 2 * i + 1, 0) % 8 for k in keys)
                    for i in range(500))
        assert ncl == 500 + stuck
        assert (label[0::2] == label[1::2]).sum() == 500 - stuck


def test_isolated_nodes_pack_into_bound_sized_groups():
    # only isolated unit nodes: ceil(n / U) clusters when the shrink cap is off
    g = isolated(1000)
    nocap = orc.Config.default(shrink_num=1000, shrink_den=1)
    for U in (2, 7, 64, 1000):
        label, ncl, _ = orc.cluster(g, U, 1, 1, nocap)
        assert ncl == math.ceil(1000 / U)
        assert _cluster_weights(g, label).max() <= U
    # with the default 2.5x cap the count stops exactly at ceil(2n/5)
    label, ncl, _ = orc.cluster(g, 64, 1, 1)
    assert ncl == math.ceil(2 * 1000 / 5) and len(np.unique(label)) == ncl


def test_star_respects_the_bound_and_theorem1():
    L, U = 300, 16
    g = star(L)
    nocap = orc.Config.default(shrink_num=1000, shrink_den=1)
    label, ncl, st = orc.cluster(g, U, 1, 5, nocap)
    w = _cluster_weights(g, label)
    assert w.max() <= U
    # Theorem 1: |C| <= |V|/2 + c(V)/U (no isolated nodes, U >= 2 c(V)/|V|)
    assert ncl <= (L + 1) / 2 + (L + 1) / U
    # after 2-hop no two light singletons share the centre's cluster as favourite
    sizes = np.bincount(label, minlength=g.n)
    assert (sizes[label[1:]] == 1).sum() <= 1


@pytest.mark.parametrize("seed", [1, 4])
def test_theorem1_bound_on_random_graphs(seed):
    g = gg.er(3000, 6000, seed)
    deg = g.degrees()
    keep = np.flatnonzero(deg > 0)
    assert len(keep) > 2500
    nocap = orc.Config.default(shrink_num=1000, shrink_den=1)
    W = g.n
    for U in (4, 16, 64):
        label, ncl, _ = orc.cluster(g, U, 1, seed, nocap)
        w = _cluster_weights(g, label)
        assert w.max() <= U
        niso = int((deg == 0).sum())
        # Theorem 1 on the non-isolated part plus the packed isolated nodes
        assert ncl <= (g.n - niso) / 2 + W / U + math.ceil(niso / (U // 1)) + 1


def test_cluster_bound_and_cap_invariants():
    g = gg.with_node_weights(gg.er(4000, 20000, 9), 3)
    n_min = math.ceil(2 * g.n / 5)
    for U in (6, 30):
        label, ncl, st = orc.cluster(g, U, 1, 3)
        w = _cluster_weights(g, label)
        heavy = g.vwgt > U
        assert (w[label[~heavy]] <= U).all()
        assert len(np.unique(label)) == ncl
        # Sec. 4.3: at most a 2.5x node reduction, exactly
        assert ncl >= n_min


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lp_cap_is_exact_when_lp_would_overshoot(seed):
    # a random graph with a generous U shrinks well past 2.5x without the cap; with it
    # the level ends at n_min clusters (plus the clusters a refill keeps alive)
    g = gg.er(6000, 30000, seed)
    n_min = math.ceil(2 * g.n / 5)
    for S in (1, 2, 8):
        cfg = orc.Config.default(lp_subrounds=S, two_hop=0, isolated=0)
        label, ncl, st = orc.cluster(g, 50, 1, seed, cfg)
        assert ncl >= n_min
        assert ncl <= n_min + g.n // 100, (S, ncl, n_min)
        assert len(np.unique(label)) == ncl
        cmap, nc, _ = orc.coarsen(g, 50, 1, seed, cfg)
        assert 5 * nc >= 2 * g.n  # n / n' <= 2.5


def test_coarsen_gives_dense_ids():
    g = gg.er(2000, 8000, 2)
    cmap, nc, _ = orc.coarsen(g, 10, 1, 1)
    assert cmap.min() == 0 and cmap.max() == nc - 1 and len(np.unique(cmap)) == nc
    label, ncl, _ = orc.cluster(g, 10, 1, 1)
    assert ncl == nc
    # rank of the label among used labels
    used = np.unique(label)
    assert (cmap == np.searchsorted(used, label)).all()


def test_no_move_rounds_stop_early():
    g = clique(6)
    k6 = hand(6, g)
    label, ncl, st = orc.cluster(k6, 6, 1, 1)
    assert ncl == 1 or ncl <= 3
    assert st.lp_subrounds <= 5 * 8


# ----------------------------------------------------------- sparsification

@pytest.mark.parametrize("wmax", [1, 3, 50])
def test_weighted_threshold_sampling_definition(wmax):
    g = gg.with_edge_weights(gg.er(3000, 30000, 5), wmax)
    m = g.m
    rows = row_index(g)
    upper = rows < g.adjncy
    w_sorted = np.sort(g.adjwgt[upper])[::-1]
    for mh in (1, 100, m // 3, m - 1):
        s, st = orc.sparsify(g, mh, 2, 7)
        check_csr(s)
        wt = int(w_sorted[mh - 1])                       # the m_hat-th heaviest edge
        assert st.omega_t == wt
        assert st.n_greater == int((w_sorted > wt).sum()) < mh <= int((w_sorted >= wt).sum())
        kept = to_sets(s)
        orig = to_sets(g)
        assert all(orig[e] == w for e, w in kept.items())            # weights unchanged
        assert all(w >= wt for w in kept.values())                    # nothing lighter kept
        heavier = {e for e, w in orig.items() if w > wt}
        assert heavier <= set(kept)                                  # all of E> kept
        assert st.threshold == ((mh - st.n_greater) << 32) // st.n_equal


def test_sparsify_extremes():
    g = gg.er(500, 2000, 1)
    s, _ = orc.sparsify(g, 0, 2, 1)
    assert s.m2 == 0 and s.n == g.n
    s, _ = orc.sparsify(g, g.m, 2, 1)
    assert to_sets(s) == to_sets(g)
    s, _ = orc.sparsify(g, 10 * g.m, 2, 1)
    assert to_sets(s) == to_sets(g)


def test_threshold_sampling_expectation_over_seeds():
    # E[kept of E=] = m_hat - |E>| (Sec. 4.2: sampled with p = (m_hat - |E>|)/|E=|)
    g = gg.with_edge_weights(gg.er(2000, 16000, 3), 4)
    mh = 5000
    kept = []
    for seed in range(64):
        s, st = orc.sparsify(g, mh, 2, seed)
        kept.append(s.m - st.n_greater)
    target = mh - st.n_greater
    p = target / st.n_equal
    sd = math.sqrt(st.n_equal * p * (1 - p)) / math.sqrt(64)
    assert abs(np.mean(kept) - target) < 4 * sd


def test_uniform_sampling_expectation():
    g = gg.er(2000, 16000, 3)
    mh = 4000
    kept = [orc.sparsify(g, mh, 2, s, mode=2)[0].m for s in range(32)]
    p = mh / g.m
    sd = math.sqrt(g.m * p * (1 - p)) / math.sqrt(32)
    assert abs(np.mean(kept) - mh) < 4 * sd


# ------------------------------------------------------------- partitioning

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("k", [2, 3])
def test_partition_not_better_than_brute_force(seed, k):
    g = gg.with_edge_weights(gg.er(11, 22, seed), 4)
    r = orc.partition(g, k, 0.03, seed)
    assert r.rc == orc.OK
    Lmax = orc.lmax(g.n, k, 30000)
    opt = brute_force_opt(g, k, Lmax)
    assert opt is not None
    assert r.cut >= opt
    assert np.bincount(r.blocks, weights=g.vwgt, minlength=k).max() <= Lmax
    assert r.cut == orc.cut(g, r.blocks)


def test_partition_hits_optimum_on_structured_graphs():
    # two K5 joined by one edge, k = 2, eps = 0.03: L_max = floor(5 * 1.03) = 5, OPT = 1
    g = hand(10, clique(5) + clique(5, 5) + [(4, 5)])
    assert brute_force_opt(g, 2, 5) == 1
    for seed in (1, 2, 3):
        r = orc.partition(g, 2, 0.03, seed)
        assert r.cut == 1
    # 4x4 grid, k = 2: OPT = 4
    grid = gg.grid2d(4, 4)
    assert brute_force_opt(grid, 2, orc.lmax(16, 2, 30000)) == 4
    r = orc.partition(grid, 2, 0.03, 1)
    assert r.cut == 4


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_partition_balance_and_cut_consistency(k):
    g = gg.er(20000, 100000, 2)
    r = orc.partition(g, k, 0.03, 1)
    assert r.rc == orc.OK
    Lmax = orc.lmax(g.n, k, 30000)
    bw = np.bincount(r.blocks, minlength=k)
    assert bw.max() <= Lmax                      # balance (Sec. 2)
    assert r.cut == orc.cut(g, r.blocks)
    assert 0 <= r.blocks.min() and r.blocks.max() < k


def test_partition_k1_and_empty():
    g = gg.er(100, 300, 1)
    r = orc.partition(g, 1, 0.03, 1)
    assert r.rc == orc.OK and r.cut == 0 and (r.blocks == 0).all()


def test_ip_and_refine_keep_balance():
    g = gg.with_node_weights(gg.grid2d(30, 30), 4)
    W = int(g.vwgt.sum())
    for k in (2, 5, 8):
        Lmax = orc.lmax(W, k, 30000)
        blk = orc.initial_partition(g, k, 30000, 3)
        assert set(np.unique(blk)) <= set(range(k))
        blk, _ = orc.rebalance(g, k, Lmax, blk)
        assert np.bincount(blk, weights=g.vwgt, minlength=k).max() <= Lmax
        ref, _ = orc.refine(g, k, Lmax, 1, 3, blk)
        assert np.bincount(ref, weights=g.vwgt, minlength=k).max() <= Lmax


def test_refinement_gains_are_positive_on_planted_blocks():
    # two dense blocks with a few cross edges, started from a noisy split:
    # LP refinement must recover a much smaller cut
    rng = np.random.default_rng(0)
    edges = []
    for off in (0, 100):
        for _ in range(800):
            a, b = rng.integers(0, 100, 2)
            if a != b:
                edges.append((off + a, off + b))
    for _ in range(20):
        edges.append((int(rng.integers(0, 100)), int(rng.integers(100, 200))))
    g = hand(200, edges)
    blk = (np.arange(200) >= 100).astype(np.int32)
    noisy = blk.copy()
    flip = rng.choice(200, 30, replace=False)
    noisy[flip] ^= 1
    Lmax = orc.lmax(200, 2, 30000)
    before = orc.cut(g, noisy)
    ref, moves = orc.refine(g, 2, Lmax, 1, 1, noisy)
    assert moves > 0 and orc.cut(g, ref) < before / 2


# ------------------------------------------------------- hierarchy invariants

def test_hierarchy_edge_bounds_on_er_c1():
    """Edge bounds of Alg. 1 per level, geometric node shrink (R13), ER triggers (Sec. 4.2)."""
    g = gg.er(65536, 524288, 1)
    r = orc.partition(g, 2, 0.03, 1)
    assert r.rc == orc.OK
    lv = r.levels()
    assert len(lv) >= 3
    cfg = orc.Config.default()
    for L in lv:
        assert L["m_next"] <= L["m_coarse"] <= L["m"]
        assert L["n_next"] * 21 <= L["n"] * 20
        assert L["m_hat"] == orc.m_hat(L["m"], L["n"], L["n_next"], cfg)
        if L["triggered"]:
            assert L["m_coarse"] > 4 * L["m_hat"]
            assert L["m_next"] <= L["m_hat"] + 6 * math.sqrt(L["m_hat"])
        else:
            assert L["m_next"] <= 4 * L["m_hat"]
    assert any(L["triggered"] for L in lv)          # low modularity: sparsification fires
    # ER expectation (Sec. 4.2): without sparsification the first contraction keeps
    # almost all edges
    assert lv[0]["m_coarse"] / lv[0]["m"] > 0.8
    # balance
    assert np.bincount(r.blocks, minlength=2).max() <= orc.lmax(65536, 2, 30000)


def test_no_sparsification_when_disabled():
    g = gg.er(20000, 100000, 1)
    r = orc.partition(g, 2, 0.03, 1, orc.Config.default(sparsifier=0))
    lv = r.levels()
    assert not any(L["triggered"] for L in lv)
    assert all(L["m_next"] == L["m_coarse"] for L in lv)


def test_determinism():
    g = gg.rmat(12, 8)
    a = orc.partition(g, 4, 0.03, 9)
    b = orc.partition(g, 4, 0.03, 9)
    assert a.cut == b.cut and (a.blocks == b.blocks).all()
    c = orc.partition(g, 4, 0.03, 10)
    assert not (a.blocks == c.blocks).all()


# ------------------------------------------- exact-count threshold sampling

def test_h64_extends_h32():
    k = orc.key(11, orc.TAG_SPARSE, 3, 0)
    for x, y in [(0, 1), (5, 77), (123456, 7654321), (2**31 - 2, 2**31 - 1)]:
        assert orc.h64(k, x, y) >> 32 == orc.h32(k, x, y)


@pytest.mark.parametrize("wmax,seed", [(1, 1), (3, 2), (50, 3)])
def test_exact_count_sampling_keeps_exactly_m_hat(wmax, seed):
    # mode 3: of the edges of weight omega_t exactly m_hat - |E>| stay, the first ones in the
    # order of (64-bit hash, min, max); the level then holds exactly m_hat edges
    g = gg.with_edge_weights(gg.er(3000, 30000, 5), wmax)
    orig = {e: w for e, w in to_sets(g).items() if e[0] < e[1]}
    for mh in (1, 100, g.m // 3, g.m - 1):
        s, st = orc.sparsify(g, mh, 2, seed, mode=3)
        check_csr(s)
        kept = {e: w for e, w in to_sets(s).items() if e[0] < e[1]}  # undirected edges
        assert len(kept) == mh
        wt = st.omega_t
        assert all(orig[e] == w and w >= wt for e, w in kept.items())
        assert {e for e, w in orig.items() if w > wt} <= set(kept)
        key = orc.key(seed, orc.TAG_SPARSE, 2, 0)
        order = lambda e: (orc.h64(key, e[0], e[1]), e[0], e[1])
        eq_kept = [order(e) for e, w in kept.items() if w == wt]
        eq_dropped = [order(e) for e, w in orig.items() if w == wt and e not in kept]
        assert len(eq_kept) == mh - st.n_greater
        if eq_kept and eq_dropped:
            assert max(eq_kept) < min(eq_dropped)
        if eq_kept:
            assert st.threshold == max(eq_kept)[0]


def test_partition_with_exact_count_sampling_meets_the_edge_bound():
    g = gg.er(20000, 100000, 3)
    r = orc.partition(g, 4, 0.03, 1, orc.Config.default(sparsifier=3))
    assert r.rc == orc.OK
    trig = [r.stats.lv[i] for i in range(r.stats.levels) if r.stats.lv[i].triggered]
    assert trig
    assert all(L.m_next == L.m_hat for L in trig)


# ----------------------------------------------------- modularity (Sec. 5)

def _modularity_direct(g, lab):
    """Q_C, sum e_ii and alpha_C of Sec. 5 from the edge list, in floating point."""
    m2 = float(np.asarray(g.adjwgt, dtype=np.float64).sum())
    rows = row_index(g)
    w = np.asarray(g.adjwgt, dtype=np.float64)
    inside = w[lab[rows] == lab[g.adjncy]].sum() / m2
    vol = np.bincount(lab[rows], weights=w, minlength=lab.max() + 1) / m2
    return inside - (vol ** 2).sum(), inside, vol.max()


def test_modularity_hand_example():
    # two triangles joined by one edge, one cluster per triangle: e_ii = 3/7, a_i = 1/2,
    # Q = 2 (3/7 - 1/4) = 5/14
    g = hand(6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (2, 3)])
    M = orc.modularity(g, np.array([0, 0, 0, 1, 1, 1]), 2)
    assert (M.w_internal, M.w_total, M.vol_max, M.vol_sq) == (12, 14, 7, 98)
    assert abs(M.q - 5 / 14) < 1e-15 and abs(M.alpha - 0.5) < 1e-15
    # one cluster: Q = 1 - 1 = 0; singletons: Q = -sum (d_v / 2m)^2
    one = orc.modularity(g, np.zeros(6, dtype=np.int32), 1)
    assert one.q == 0.0 and one.inside == 1.0
    single = orc.modularity(g, np.arange(6), 6)
    deg = np.diff(g.xadj)
    assert abs(single.q + ((deg / 14.0) ** 2).sum()) < 1e-15


def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    for g in (gg.er(400, 1600, 2), gg.with_edge_weights(gg.er(300, 1500, 4), 9), gg.grid2d(20, 15)):
        lab, _, _ = orc.cluster(g, 8, 1, 3)
        _, lab = np.unique(lab, return_inverse=True)
        M = orc.modularity(g, lab, int(lab.max()) + 1)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        rows = row_index(g)
        for u, v, w in zip(rows.tolist(), g.adjncy.tolist(), g.adjwgt.tolist()):
            if u < v:
                G.add_edge(u, v, weight=w)
        comms = [set(np.flatnonzero(lab == c).tolist()) for c in range(int(lab.max()) + 1)]
        assert abs(M.q - nx.community.modularity(G, comms, weight="weight")) < 1e-12


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_modularity_lemma2_bounds(seed):
    # Lemma 2: Q_C <= sum_i e_ii <= Q_C + alpha_C, on LP clusterings and random ones
    g = gg.with_edge_weights(gg.er(2000, 12000, seed), 5)
    rng = np.random.default_rng(seed)
    lab_lp, _, _ = orc.cluster(g, 30, 1, seed)
    for lab in (np.unique(lab_lp, return_inverse=True)[1], rng.integers(0, 7, g.n), rng.integers(0, 500, g.n)):
        M = orc.modularity(g, lab, int(lab.max()) + 1)
        q, inside, alpha = _modularity_direct(g, lab)
        assert abs(M.q - q) < 1e-12 and abs(M.inside - inside) < 1e-12 and abs(M.alpha - alpha) < 1e-12
        assert M.q <= M.inside + 1e-15 <= M.q + M.alpha + 2e-15
        assert 1 - M.inside >= M.bound - 1e-15  # the between-cluster fraction exceeds the bound


def test_modularity_rejects_labels_out_of_range():
    g = gg.er(100, 300, 1)
    with pytest.raises(RuntimeError):
        orc.modularity(g, np.full(g.n, 3), 3)
