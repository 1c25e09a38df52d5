"""Hand-traced pins of the oracle's schedule readings (tests/golden/schedule_pins.txt).

The fixture holds small graphs whose outcome under the readings R6 (tie-breaking),
R7 (longest-prefix acceptance), R8 (the exact 2.5x cap of Sec. 4.3), R18 (batched
greedy growing with frozen gains) and R19 (greedy rebalance) was worked out by hand.
Each case is run through the oracle and compared with the traced result; every hash
value the trace relies on is re-checked against the oracle's hash, which is itself
pinned to the published SplitMix64 vectors.  A plausible mistake in any of these
readings (accepting whatever fits, max instead of min loss, counting refilled clusters,
updating gains inside a growing step, ...) changes one of the traced results.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "schedule_pins.txt")


def load_cases(path=FIXTURE):
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].rstrip() if not raw.lstrip().startswith("#") else ""
            if not line.strip():
                continue
            key, _, val = line.partition(":")
            key, val = key.strip(), val.strip()
            if key == "case":
                cur = {"case": val, "hash": []}
                cases.append(cur)
            elif key == "hash":
                cur["hash"].append(val)
            else:
                cur[key] = val
    return cases


CASES = load_cases()


def graph_of(c):
    n = int(c["n"])
    u, v, w = [], [], []
    for tok in c.get("edges", "").split():
        ends, _, wt = tok.partition(":")
        a, b = ends.split("-")
        u.append(int(a)); v.append(int(b)); w.append(int(wt))
    g = gg.from_pairs(n, u, v, name=c["case"])
    wmap = {(min(a, b), max(a, b)): x for a, b, x in zip(u, v, w)}
    rows = np.repeat(np.arange(n), np.diff(g.xadj))
    g.adjwgt = np.array([wmap[(min(int(r), int(q)), max(int(r), int(q)))]
                         for r, q in zip(rows, g.adjncy)], dtype=np.int32)
    vw = np.ones(n, dtype=np.int32)
    for tok in c.get("vwgt", "").split():
        a, _, x = tok.partition(":")
        vw[int(a)] = int(x)
    g.vwgt = vw
    return g


def config_of(c):
    cfg = orc.Config.default()
    for tok in c.get("cfg", "").split():
        name, _, val = tok.partition("=")
        setattr(cfg, name, int(val))
    return cfg


def ints(s):
    return [int(x) for x in s.split()]


def check_hashes(c):
    S = config_of(c).lp_subrounds
    for h in c["hash"]:
        lhs, _, rhs = h.partition("=")
        f = lhs.split()
        if f[0] == "h32":
            seed, tag, level, rnd, x, y = (int(t) for t in f[1:])
            assert orc.h32(orc.key(seed, tag, level, rnd), x, y) == int(rhs, 0), h
        elif f[0] == "act":
            seed, tag, level, rnd = (int(t) for t in f[1:])
            k = orc.key(seed, tag, level, rnd)
            want = ints(rhs)
            assert [orc.h32(k, v, 0) % S for v in range(len(want))] == want, h
        else:
            raise AssertionError(f"unknown hash record {h}")
    if "hash_min" in c:
        lhs, _, rhs = c["hash_min"].partition("=")
        seed, tag, level, rnd, t, nv = (int(x) for x in lhs.split())
        k = orc.key(seed, tag, level, rnd)
        assert min(range(nv), key=lambda v: (orc.h32(k, v, t), v)) == int(rhs)


@pytest.mark.parametrize("c", CASES, ids=[c["case"] for c in CASES])
def test_schedule_pin(c):
    check_hashes(c)
    g = graph_of(c)
    call = c["call"]
    if call == "cluster":
        label, ncl, st = orc.cluster(g, int(c["U"]), int(c["level"]), int(c["seed"]), config_of(c))
        if "expect_label" in c:
            assert label.tolist() == ints(c["expect_label"])
        for tok in c.get("expect_label_at", "").split():
            v, _, lab = tok.partition(":")
            assert int(label[int(v)]) == int(lab), tok
        if "expect_nclusters" in c:
            assert ncl == int(c["expect_nclusters"])
            assert len(np.unique(label)) == ncl
        if "expect_subrounds" in c:
            assert st.lp_subrounds == int(c["expect_subrounds"])
        assert st.lp_moves == int(c["expect_moves"])
    elif call == "refine":
        blk, moves = orc.refine(g, int(c["k"]), int(c["Lmax"]), int(c["level"]), int(c["seed"]),
                                np.array(ints(c["blocks"]), dtype=np.int32), config_of(c))
        assert blk.tolist() == ints(c["expect_blocks"])
        assert moves == int(c["expect_moves"])
    elif call == "rebalance":
        blk, moves = orc.rebalance(g, int(c["k"]), int(c["Lmax"]),
                                   np.array(ints(c["blocks"]), dtype=np.int32))
        assert blk.tolist() == ints(c["expect_blocks"])
        assert moves == int(c["expect_moves"])
    elif call == "initial_partition":
        blk = orc.initial_partition(g, int(c["k"]), int(c["eps_ppm"]), int(c["seed"]),
                                    int(c["trials"]))
        side = set(ints(c["expect_block0"]))
        want = np.array([0 if v in side else 1 for v in range(g.n)], dtype=np.int32)
        assert (blk == want).all(), sorted(np.flatnonzero(blk == 0).tolist())[:20]
    else:
        raise AssertionError(f"unknown call {call}")


def test_fixture_covers_every_reading():
    names = {c["case"] for c in CASES}
    for prefix in ("r6_", "r7_", "r8_", "r18_", "r19_"):
        assert any(n.startswith(prefix) for n in names), prefix
