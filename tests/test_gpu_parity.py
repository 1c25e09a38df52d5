"""GPU (C-ABI) vs CPU oracle parity, element by element.

Integer work with a fixed deterministic schedule: every comparison is exact
(tolerance 0).  Coarse rows come back from the GPU in unspecified order, so
graphs are compared row by row after sorting each row.  Inputs are chosen to
exercise every kernel variant: degrees <= 32 (warp, one neighbour per lane),
33..128 (warp hash table), 129..2048 (block, shared table), > 2048 (block,
global table), isolated nodes, node and edge weights, several tiles and
ragged tails.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen as gg
import oracle as orc
from tests._util import clique, hand, matching, star

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


def _graphs():
    return {
        "er": gg.er(3000, 15000, 1),
        "er_w": gg.with_node_weights(gg.with_edge_weights(gg.er(5000, 40000, 2), 7), 3),
        "rmat12": gg.rmat(12, 8, seed=3),
        "grid": gg.grid2d(60, 50),
        "star": star(3000),
        "matching": matching(2000),
        "iso": gg.with_isolated(gg.er(2000, 6000, 4), 700),
        "dense": gg.er(600, 60000, 5),
    }


GRAPHS = _graphs()


def canon(g):
    """(xadj, rows sorted) as numpy arrays for exact comparison."""
    xadj = np.asarray(g.xadj, dtype=np.int64)
    adj = np.asarray(g.adjncy, dtype=np.int64).copy()
    w = np.asarray(g.adjwgt, dtype=np.int64).copy()
    for v in range(g.n):
        a, b = xadj[v], xadj[v + 1]
        if b - a > 1:
            o = np.argsort(adj[a:b], kind="stable")
            adj[a:b] = adj[a:b][o]
            w[a:b] = w[a:b][o]
    return xadj, adj, w, np.asarray(g.vwgt, dtype=np.int64)[:g.n]


def assert_same_graph(got, exp):
    gx, ga, gw, gv = canon(got)
    ex, ea, ew, ev = canon(exp)
    assert got.n == exp.n
    assert np.array_equal(gv, ev), "node weights differ"
    assert np.array_equal(gx, ex), "row offsets differ"
    assert np.array_equal(ga, ea), "neighbours differ"
    assert np.array_equal(gw, ew), "edge weights differ"


def _level_fields(st):
    return (st.lp_subrounds, st.lp_moves, st.clusters_lp, st.clusters_2hop, st.clusters_final, st.n_next)


# --------------------------------------------------------------- coarsening

@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("seed", [1, 7])
def test_coarsen_matches_oracle(gp, ctx, name, seed):
    g = GRAPHS[name]
    W = int(g.vwgt.sum())
    for U in (max(1, W // (160 * 2)), 6):
        dg = gp.DeviceGraph.from_host(g)
        cmap, nc, st, label = ctx.gp_coarsen(dg, U, 1, seed, want_label=True)
        olabel, oncl, ost = orc.cluster(g, U, 1, seed)
        ocmap, onc, _ = orc.coarsen(g, U, 1, seed)
        assert np.array_equal(label.cpu().numpy(), olabel), f"labels differ ({name}, U={U})"
        assert nc == onc
        assert np.array_equal(cmap.cpu().numpy(), ocmap)
        assert (st.lp_subrounds, st.lp_moves, st.clusters_lp, st.clusters_2hop, st.clusters_final) == \
            (ost.lp_subrounds, ost.lp_moves, ost.clusters_lp, ost.clusters_2hop, ost.clusters_final)


@pytest.mark.parametrize("subs", [0, 1, 2, 3, 7, 9, 17])
def test_lp_state_after_each_subround(gp, ctx, subs):
    g = GRAPHS["er_w"]
    cfg_g = gp.default_config(dbg_max_subrounds=subs, two_hop=0, isolated=0)
    cfg_o = orc.Config.default(dbg_max_subrounds=subs, two_hop=0, isolated=0)
    dg = gp.DeviceGraph.from_host(g)
    for U in (5, 40):
        _, nc, st, label = ctx.gp_coarsen(dg, U, 2, 3, cfg_g, want_label=True)
        olabel, oncl, ost = orc.cluster(g, U, 2, 3, cfg_o)
        assert np.array_equal(label.cpu().numpy(), olabel)
        assert nc == oncl and st.lp_subrounds == ost.lp_subrounds


def test_coarsen_config_variants(gp, ctx):
    g = GRAPHS["iso"]
    for kw in ({"two_hop": 0}, {"isolated": 0}, {"lp_subrounds": 1}, {"lp_subrounds": 3, "lp_rounds": 2},
               {"shrink_num": 1000, "shrink_den": 1}, {"lp_rounds": 0}):
        dg = gp.DeviceGraph.from_host(g)
        cmap, nc, st = ctx.gp_coarsen(dg, 9, 4, 11, gp.default_config(**kw))
        ocmap, onc, _ = orc.coarsen(g, 9, 4, 11, orc.Config.default(**kw))
        assert nc == onc and np.array_equal(cmap.cpu().numpy(), ocmap), kw


def test_coarsen_tiny_and_degenerate(gp, ctx):
    cases = [hand(1, []), hand(2, [(0, 1)]), hand(3, []), hand(5, clique(5)), star(1),
             hand(4, [(0, 1), (2, 3)], weights=[5, 1], vwgt=[3, 1, 2, 2])]
    for g in cases:
        for U in (1, 2, 100):
            dg = gp.DeviceGraph.from_host(g)
            cmap, nc, st = ctx.gp_coarsen(dg, U, 1, 1)
            ocmap, onc, _ = orc.coarsen(g, U, 1, 1)
            assert nc == onc and np.array_equal(cmap.cpu().numpy(), ocmap)


# -------------------------------------------------------------- contraction

@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_contract_matches_oracle(gp, ctx, name):
    g = GRAPHS[name]
    ocmap, onc, _ = orc.coarsen(g, 8, 1, 1)
    rng = np.random.default_rng(5)
    rcmap = rng.integers(0, max(1, g.n // 3), g.n).astype(np.int32)
    used = np.unique(rcmap)
    rcmap = np.searchsorted(used, rcmap).astype(np.int32)
    cmaps = [(ocmap, onc), (rcmap, len(used)), (np.zeros(g.n, np.int32), 1)]
    import torch
    for cmap, nc in cmaps:
        dg = gp.DeviceGraph.from_host(g)
        out = ctx.gp_contract(dg, torch.from_numpy(cmap).cuda(), nc)
        got = out.to_host()
        exp = orc.contract(g, cmap, nc)
        assert_same_graph(got, exp)
        out.release()


# ----------------------------------------------------------- sparsification

@pytest.mark.parametrize("wmax", [1, 5, 100000])
@pytest.mark.parametrize("mode", [1, 2, 3])
def test_sparsify_matches_oracle(gp, ctx, wmax, mode):
    g = gg.with_edge_weights(gg.er(4000, 50000, 6), wmax)
    dg = gp.DeviceGraph.from_host(g)
    m = g.m
    for mh in (0, 1, 3, m // 7, m // 2, m - 1, m, 2 * m):
        out, st = ctx.gp_sparsify(dg, mh, 3, 9, mode)
        exp, ost = orc.sparsify(g, mh, 3, 9, mode)
        assert_same_graph(out.to_host(), exp)
        assert (st.omega_t, st.n_greater, st.n_equal, st.threshold) == \
            (ost.omega_t, ost.n_greater, ost.n_equal, ost.threshold)
        out.release()


def test_sparsify_heavy_hub_rows(gp, ctx):
    g = gg.with_edge_weights(gg.rmat(13, 16, seed=2), 9)
    dg = gp.DeviceGraph.from_host(g)
    for mh in (g.m // 5, g.m // 2):
        out, st = ctx.gp_sparsify(dg, mh, 2, 4, 1)
        exp, ost = orc.sparsify(g, mh, 2, 4, 1)
        assert_same_graph(out.to_host(), exp)
        out.release()


# ---------------------------------------------- initial partition, balance

def _coarse(g, levels=2, k=4):
    cur = g
    W = int(g.vwgt.sum())
    U = orc.cluster_bound(W, k)
    for i in range(levels):
        cmap, nc, _ = orc.coarsen(cur, U, i + 1, 1)
        cur = orc.contract(cur, cmap, nc)
    return cur


@pytest.mark.parametrize("k", [2, 3, 4, 8, 16])
def test_initial_partition_matches_oracle(gp, ctx, k):
    for g in (_coarse(GRAPHS["er_w"]), _coarse(GRAPHS["grid"]), GRAPHS["star"], _coarse(GRAPHS["rmat12"])):
        dg = gp.DeviceGraph.from_host(g)
        blk = ctx.gp_initial_partition(dg, k, 0.03, 5)
        oblk = orc.initial_partition(g, k, 30000, 5)
        assert np.array_equal(blk.cpu().numpy(), oblk)


def test_initial_partition_large_subproblem_uses_global_state(gp, ctx):
    g = gg.er(45000, 130000, 8)   # above the shared-memory node limit (about 31k nodes)
    dg = gp.DeviceGraph.from_host(g)
    blk = ctx.gp_initial_partition(dg, 2, 0.03, 2, gp.default_config(ip_trials=2))
    oblk = orc.initial_partition(g, 2, 30000, 2, trials=2)
    assert np.array_equal(blk.cpu().numpy(), oblk)


@pytest.mark.parametrize("name", ["er", "er_heavy", "grid", "star", "rmat"])
def test_initial_partition_steps_of_many_nodes_match_oracle(gp, ctx, name):
    """Subproblems of 8k-30k nodes (growing steps of B = 8..30 nodes, selected together): plain
    ER (24k nodes: state in shared memory, fallback hashes not); ER with node weights up to 5000 (nodes that no longer fit are retired mid-step); a grid
    (many equal gains); a star (after the centre every leaf has the same gain, so the candidates
    overflow the ranked set and the step falls back to one-by-one extraction); R-MAT."""
    g = {"er": lambda: gg.er(24000, 100000, 21),
         "er_heavy": lambda: gg.with_node_weights(gg.er(16000, 70000, 22), 5000),
         "grid": lambda: gg.grid2d(110, 100),
         "star": lambda: star(10000),
         "rmat": lambda: gg.rmat(14, 6, seed=23)}[name]()
    dg = gp.DeviceGraph.from_host(g)
    for k, trials in ((2, 3), (5, 2)):
        blk = ctx.gp_initial_partition(dg, k, 0.03, 9, gp.default_config(ip_trials=trials))
        oblk = orc.initial_partition(g, k, 30000, 9, trials=trials)
        assert np.array_equal(blk.cpu().numpy(), oblk), (name, k)


@pytest.mark.parametrize("k", [2, 5, 8])
def test_rebalance_matches_oracle(gp, ctx, k):
    import torch
    g = gg.with_node_weights(gg.grid2d(40, 40), 4)
    W = int(g.vwgt.sum())
    Lmax = orc.lmax(W, k, 30000)
    rng = np.random.default_rng(k)
    blk = np.where(rng.random(g.n) < 0.6, 0, rng.integers(0, k, g.n)).astype(np.int32)
    dg = gp.DeviceGraph.from_host(g)
    t = torch.from_numpy(blk.copy()).cuda()
    mv = ctx.gp_rebalance(dg, k, Lmax, t)
    oblk, omv = orc.rebalance(g, k, Lmax, blk)
    assert mv == omv
    assert np.array_equal(t.cpu().numpy(), oblk)


@pytest.mark.parametrize("k", [2, 4, 16, 64, 128, 200, 300])
def test_refine_matches_oracle(gp, ctx, k):
    import torch
    for g in (GRAPHS["er_w"], GRAPHS["rmat12"], GRAPHS["grid"]):
        W = int(g.vwgt.sum())
        Lmax = orc.lmax(W, k, 30000)
        rng = np.random.default_rng(k)
        blk = rng.integers(0, k, g.n).astype(np.int32)
        blk, _ = orc.rebalance(g, k, Lmax, blk)
        dg = gp.DeviceGraph.from_host(g)
        t = torch.from_numpy(blk.copy()).cuda()
        mv = ctx.gp_refine(dg, k, Lmax, 2, 13, t)
        oblk, omv = orc.refine(g, k, Lmax, 2, 13, blk)
        assert mv == omv
        assert np.array_equal(t.cpu().numpy(), oblk)


def test_cut_and_project(gp, ctx):
    import torch
    g = GRAPHS["er_w"]
    k = 7
    blk = np.random.default_rng(1).integers(0, k, g.n).astype(np.int32)
    dg = gp.DeviceGraph.from_host(g)
    cut, bw = ctx.gp_cut(dg, torch.from_numpy(blk).cuda(), k)
    assert cut == orc.cut(g, blk)
    assert np.array_equal(bw, np.bincount(blk, weights=g.vwgt, minlength=k).astype(np.int64))
    cmap = np.random.default_rng(2).integers(0, 100, g.n).astype(np.int32)
    coarse = np.random.default_rng(3).integers(0, k, 100).astype(np.int32)
    fine = ctx.gp_project(torch.from_numpy(cmap).cuda(), torch.from_numpy(coarse).cuda(), g.n)
    assert np.array_equal(fine.cpu().numpy(), coarse[cmap])


# ---------------------------------------------------------------- partition

def _check_partition(gp, ctx, g, k, eps, seed, cfg_kw=None, gpu_kw=None):
    cfg_kw = cfg_kw or {}
    dg = gp.DeviceGraph.from_host(g)
    blocks, cut, st = ctx.gp_partition(dg, k, eps, seed, gp.default_config(**cfg_kw, **(gpu_kw or {})))
    r = orc.partition(g, k, eps, seed, orc.Config.default(**cfg_kw))
    assert r.rc == orc.OK
    assert cut == r.cut
    assert np.array_equal(blocks.cpu().numpy(), r.blocks)
    assert st.levels == r.stats.levels
    for a, b in zip([st.lv[i] for i in range(st.levels)], [r.stats.lv[i] for i in range(r.stats.levels)]):
        for f in ("n", "n_next", "m", "m_coarse", "m_hat", "m_next", "triggered", "omega_t",
                  "n_greater", "n_equal", "threshold", "lp_subrounds", "lp_moves", "clusters_lp",
                  "clusters_2hop", "clusters_final"):
            assert getattr(a, f) == getattr(b, f), f
    assert (st.U, st.Lmax, st.W, st.ip_cut, st.rebalance_moves, st.n_coarsest) == \
        (r.stats.U, r.stats.Lmax, r.stats.W, r.stats.ip_cut, r.stats.rebalance_moves, r.stats.n_coarsest)
    assert np.bincount(r.blocks, weights=g.vwgt, minlength=k).max() <= st.Lmax
    return st


def test_partition_er_c1_matches_oracle(gp, ctx):
    g = gg.er(65536, 524288, 1)
    st = _check_partition(gp, ctx, g, 2, 0.03, 1)
    assert any(st.lv[i].triggered for i in range(st.levels))


@pytest.mark.parametrize("name,k", [("er", 4), ("er_w", 8), ("rmat12", 16), ("grid", 3), ("iso", 5),
                                    ("star", 2), ("dense", 6), ("matching", 4)])
def test_partition_matches_oracle(gp, ctx, name, k):
    _check_partition(gp, ctx, GRAPHS[name], k, 0.03, 2)


@pytest.mark.parametrize("kw", [{"sparsifier": 0}, {"sparsifier": 2}, {"sparsifier": 3}, {"ref_rounds": 0},
                                {"coarsest_factor": 20}, {"ip_trials": 1}])
def test_partition_config_variants(gp, ctx, kw):
    _check_partition(gp, ctx, gg.er(20000, 100000, 3), 4, 0.05, 4, kw)


def test_partition_rmat_scale15(gp, ctx):
    _check_partition(gp, ctx, gg.rmat(15, 16, seed=1), 64, 0.03, 1)


@pytest.mark.parametrize("k", [129, 256, 300])
def test_partition_many_blocks(gp, ctx, k):
    # narrow (uint8) and wide block ids in refinement and the cut
    _check_partition(gp, ctx, gg.er(60000, 300000, 7), k, 0.03, 3)


def test_partition_host_entry_matches_device(gp, ctx):
    g = GRAPHS["er_w"]
    dg = gp.DeviceGraph.from_host(g)
    blocks, cut, st = ctx.gp_partition(dg, 4, 0.03, 3)
    hb, hcut, hst = ctx.gp_partition_host(g.n, g.m2, g.xadj.astype(np.int32), g.adjncy, g.vwgt, g.adjwgt,
                                          4, 0.03, 3)
    assert hcut == cut
    assert np.array_equal(hb[:g.n], blocks.cpu().numpy())


def test_partition_trivial_cases(gp, ctx):
    g = GRAPHS["er"]
    dg = gp.DeviceGraph.from_host(g)
    blocks, cut, _ = ctx.gp_partition(dg, 1, 0.03, 1)
    assert cut == 0 and (blocks.cpu().numpy() == 0).all()
    two_k5 = hand(10, clique(5) + clique(5, 5) + [(4, 5)])
    b, c, _ = ctx.gp_partition(gp.DeviceGraph.from_host(two_k5), 2, 0.03, 1)
    assert c == 1
    e = hand(1, [])
    b, c, _ = ctx.gp_partition(gp.DeviceGraph.from_host(e), 3, 0.03, 1)
    assert c == 0


def test_validation_errors(gp, ctx):
    g = hand(4, [(0, 1), (1, 2), (2, 3)])
    bad_w = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    bad_w.adjwgt[0] = 5
    loop = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    loop.adjncy[0] = 0
    zero = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), g.adjwgt.copy())
    zero.vwgt[1] = 0
    heavy = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), np.array([1, 1, 1, 9], np.int32), g.adjwgt.copy())
    big = gg.Graph(g.n, g.xadj.copy(), g.adjncy.copy(), g.vwgt.copy(), np.full(g.m2, 2**30, np.int32))
    for bad, status in ((bad_w, gp.GP_ERR_INVALID), (loop, gp.GP_ERR_INVALID), (zero, gp.GP_ERR_INVALID),
                        (heavy, gp.GP_ERR_INFEASIBLE), (big, gp.GP_ERR_OVERFLOW)):
        with pytest.raises(gp.GpError) as ei:
            ctx.gp_partition(gp.DeviceGraph.from_host(bad), 2, 0.03, 1)
        assert ei.value.status == status
    with pytest.raises(gp.GpError):
        ctx.gp_partition(gp.DeviceGraph.from_host(g), 0, 0.03, 1)
    with pytest.raises(gp.GpError):
        ctx.gp_partition(gp.DeviceGraph.from_host(g), 2, 0.0, 1)
    # the context stays usable after errors
    blocks, cut, _ = ctx.gp_partition(gp.DeviceGraph.from_host(g), 2, 0.03, 1)
    assert cut == orc.partition(g, 2, 0.03, 1).cut


def test_partition_through_torch_allocator(gp):
    """The same partition when device memory comes from torch's caching allocator."""
    c = gp.Context(0, use_torch_allocator=True)
    try:
        g = GRAPHS["er_w"]
        dg = gp.DeviceGraph.from_host(g)
        blocks, cut, _ = c.gp_partition(dg, 8, 0.03, 2)
        r = orc.partition(g, 8, 0.03, 2)
        assert cut == r.cut and np.array_equal(blocks.cpu().numpy(), r.blocks)
    finally:
        c.close()


# ------------------------------------------------------- modularity (Sec. 5)

@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_modularity_matches_oracle(gp, ctx, name):
    import torch
    g = GRAPHS[name]
    rng = np.random.default_rng(4)
    lab_lp, _, _ = orc.cluster(g, 12, 1, 2)
    cases = [np.unique(lab_lp, return_inverse=True)[1], np.zeros(g.n, dtype=np.int64),
             np.arange(g.n), rng.integers(0, 37, g.n)]
    dg = gp.DeviceGraph.from_host(g)
    for lab in cases:
        nl = int(lab.max()) + 1
        st = ctx.gp_modularity(dg, torch.from_numpy(lab.astype(np.int32)).cuda(), nl)
        M = orc.modularity(g, lab, nl)
        assert (st.w_internal, st.w_total, st.vol_max, st.vol_sq) == (M.w_internal, M.w_total, M.vol_max, M.vol_sq)
        for f in ("inside", "q", "alpha", "bound"):
            assert abs(getattr(st, f) - getattr(M, f)) <= 1e-12, f


def test_modularity_rejects_labels_out_of_range(gp, ctx):
    import torch
    g = GRAPHS["er"]
    dg = gp.DeviceGraph.from_host(g)
    lab = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    lab[17] = 5
    with pytest.raises(gp.GpError):
        ctx.gp_modularity(dg, lab, 5)


# ------------------------------------------------- hand-traced schedule pins

from tests.test_schedule_pins import CASES as PIN_CASES, config_of, graph_of, ints  # noqa: E402


@pytest.mark.parametrize("c", PIN_CASES, ids=[c["case"] for c in PIN_CASES])
def test_schedule_pins_on_gpu(gp, ctx, c):
    """The GPU reaches the hand-traced results of the schedule readings (R6, R7, R8,
    R18, R19) through the C-ABI, and agrees with the oracle on them."""
    import torch
    g = graph_of(c)
    kw = {k: getattr(config_of(c), k) for k in ("lp_rounds", "lp_subrounds", "ref_rounds", "ip_trials",
                                                 "two_hop", "isolated", "dbg_max_subrounds")}
    if "trials" in c:
        kw["ip_trials"] = int(c["trials"])
    cfg = gp.default_config(**kw)
    dg = gp.DeviceGraph.from_host(g)
    call = c["call"]
    if call == "cluster":
        _, nc, st, label = ctx.gp_coarsen(dg, int(c["U"]), int(c["level"]), int(c["seed"]), cfg,
                                          want_label=True)
        label = label.cpu().numpy()
        if "expect_label" in c:
            assert label.tolist() == ints(c["expect_label"])
        for tok in c.get("expect_label_at", "").split():
            v, _, lab = tok.partition(":")
            assert int(label[int(v)]) == int(lab), tok
        if "expect_nclusters" in c:
            assert nc == int(c["expect_nclusters"])
        if "expect_subrounds" in c:
            assert st.lp_subrounds == int(c["expect_subrounds"])
        assert st.lp_moves == int(c["expect_moves"])
    elif call in ("refine", "rebalance"):
        blk = torch.tensor(ints(c["blocks"]), dtype=torch.int32, device="cuda")
        if call == "refine":
            mv = ctx.gp_refine(dg, int(c["k"]), int(c["Lmax"]), int(c["level"]), int(c["seed"]), blk, cfg)
        else:
            mv = ctx.gp_rebalance(dg, int(c["k"]), int(c["Lmax"]), blk)
        assert blk.cpu().numpy().tolist() == ints(c["expect_blocks"])
        assert mv == int(c["expect_moves"])
    elif call == "initial_partition":
        blk = ctx.gp_initial_partition(dg, int(c["k"]), int(c["eps_ppm"]) / 1e6, int(c["seed"]), cfg)
        side = set(ints(c["expect_block0"]))
        want = np.array([0 if v in side else 1 for v in range(g.n)], dtype=np.int32)
        assert np.array_equal(blk.cpu().numpy(), want)
    else:
        raise AssertionError(call)


# ------------------------------------- both LP drivers: persistent and per-phase
#
# Graphs up to gp_config.small_lp_nodes nodes run each LP call as one persistent
# launch (every test above on small graphs goes that way by default);
# small_lp_nodes = 0 forces the per-phase driver that large levels use.

HOST_PATH = dict(small_lp_nodes=0)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_coarsen_per_phase_driver_matches_oracle(gp, ctx, name):
    g = GRAPHS[name]
    W = int(g.vwgt.sum())
    for U in (max(1, W // (160 * 2)), 6):
        dg = gp.DeviceGraph.from_host(g)
        cmap, nc, st, label = ctx.gp_coarsen(dg, U, 1, 7, gp.default_config(**HOST_PATH), want_label=True)
        olabel, oncl, ost = orc.cluster(g, U, 1, 7)
        assert np.array_equal(label.cpu().numpy(), olabel), f"labels differ ({name}, U={U})"
        assert (st.lp_subrounds, st.lp_moves, st.clusters_lp, st.clusters_final) == \
            (ost.lp_subrounds, ost.lp_moves, ost.clusters_lp, ost.clusters_final)


@pytest.mark.parametrize("subs", [1, 3, 9])
def test_lp_state_per_phase_driver(gp, ctx, subs):
    g = GRAPHS["er_w"]
    kw = dict(dbg_max_subrounds=subs, two_hop=0, isolated=0)
    dg = gp.DeviceGraph.from_host(g)
    for U in (5, 40):
        _, nc, st, label = ctx.gp_coarsen(dg, U, 2, 3, gp.default_config(**kw, **HOST_PATH), want_label=True)
        olabel, oncl, ost = orc.cluster(g, U, 2, 3, orc.Config.default(**kw))
        assert np.array_equal(label.cpu().numpy(), olabel)
        assert nc == oncl and st.lp_subrounds == ost.lp_subrounds


@pytest.mark.parametrize("k", [2, 128, 300])
def test_refine_per_phase_driver_matches_oracle(gp, ctx, k):
    import torch
    for g in (GRAPHS["er_w"], GRAPHS["rmat12"]):
        Lmax = orc.lmax(int(g.vwgt.sum()), k, 30000)
        blk = np.random.default_rng(k).integers(0, k, g.n).astype(np.int32)
        blk, _ = orc.rebalance(g, k, Lmax, blk)
        dg = gp.DeviceGraph.from_host(g)
        t = torch.from_numpy(blk.copy()).cuda()
        mv = ctx.gp_refine(dg, k, Lmax, 2, 13, t, gp.default_config(**HOST_PATH))
        oblk, omv = orc.refine(g, k, Lmax, 2, 13, blk)
        assert mv == omv and np.array_equal(t.cpu().numpy(), oblk)


@pytest.mark.parametrize("name,k", [("er", 4), ("rmat12", 16), ("star", 2), ("dense", 6)])
def test_partition_per_phase_driver_matches_oracle(gp, ctx, name, k):
    _check_partition(gp, ctx, GRAPHS[name], k, 0.03, 2, gpu_kw=HOST_PATH)


def test_partition_both_drivers_agree_on_c1(gp, ctx):
    g = gg.er(65536, 524288, 1)
    dg = gp.DeviceGraph.from_host(g)
    b1, c1, s1 = ctx.gp_partition(dg, 2, 0.03, 1)
    b2, c2, s2 = ctx.gp_partition(dg, 2, 0.03, 1, gp.default_config(**HOST_PATH))
    assert c1 == c2 and np.array_equal(b1.cpu().numpy(), b2.cpu().numpy())


def test_persistent_lp_wait_limit_gives_timeout_and_context_survives(gp, ctx):
    """A grid-wide wait of the persistent LP kernel that runs out returns GP_ERR_TIMEOUT
    (no trap, no hang); the context then works as before."""
    g = GRAPHS["er"]
    dg = gp.DeviceGraph.from_host(g)
    ctx.gp_set_wait_limit(-1)  # every device-side wait gives up at once
    try:
        with pytest.raises(gp.GpError) as ei:
            ctx.gp_coarsen(dg, 20, 1, 1)
        assert ei.value.status == gp.GP_ERR_TIMEOUT
    finally:
        ctx.gp_set_wait_limit(0)
    cmap, nc, _ = ctx.gp_coarsen(dg, 20, 1, 1)
    ocmap, onc, _ = orc.coarsen(g, 20, 1, 1)
    assert nc == onc and np.array_equal(cmap.cpu().numpy(), ocmap)
