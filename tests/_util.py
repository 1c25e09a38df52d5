"""Small helpers shared by the tests: hand-made graphs and checks on CSR graphs."""
from __future__ import annotations

import itertools

import numpy as np

import graphgen as gg


def hand(n, edges, weights=None, vwgt=None, name="hand"):
    """Graph from an undirected edge list; weights given per listed edge."""
    u = [a for a, _ in edges]
    v = [b for _, b in edges]
    g = gg.from_pairs(n, u, v, name=name)
    if weights is not None:
        wmap = {}
        for (a, b), w in zip(edges, weights):
            wmap[(min(a, b), max(a, b))] = w
        rows = g.rows()
        aw = np.array([wmap[(min(int(r), int(c)), max(int(r), int(c)))]
                       for r, c in zip(rows, g.adjncy)], dtype=np.int32)
        g.adjwgt = aw
    if vwgt is not None:
        g.vwgt = np.asarray(vwgt, dtype=np.int32)
    return g


def path(n):
    return hand(n, [(i, i + 1) for i in range(n - 1)], name=f"path{n}")


def clique(n, offset=0):
    return [(offset + i, offset + j) for i in range(n) for j in range(i + 1, n)]


def star(leaves):
    return hand(leaves + 1, [(0, i) for i in range(1, leaves + 1)], name=f"star{leaves}")


def matching(pairs):
    return hand(2 * pairs, [(2 * i, 2 * i + 1) for i in range(pairs)], name=f"matching{pairs}")


def isolated(n):
    return hand(n, [], name=f"isolated{n}")


def to_sets(g):
    """{(u, v): w} over all CSR entries."""
    rows = g.rows() if hasattr(g, "rows") else np.repeat(np.arange(g.n), np.diff(g.xadj))
    return {(int(r), int(c)): int(w) for r, c, w in zip(rows, g.adjncy, g.adjwgt)}


def row_index(g):
    return np.repeat(np.arange(g.n, dtype=np.int64), np.diff(np.asarray(g.xadj, dtype=np.int64)))


def check_csr(g, sorted_rows=True):
    """Symmetric, loop-free, duplicate-free, positive weights."""
    xadj = np.asarray(g.xadj, dtype=np.int64)
    assert xadj[0] == 0 and (np.diff(xadj) >= 0).all()
    rows = row_index(g)
    adj = np.asarray(g.adjncy, dtype=np.int64)
    assert (adj != rows).all(), "self-loop"
    assert ((adj >= 0) & (adj < g.n)).all()
    assert (np.asarray(g.adjwgt) > 0).all()
    fwd = rows * g.n + adj
    rev = adj * g.n + rows
    assert len(np.unique(fwd)) == len(fwd), "duplicate entry"
    order = np.argsort(fwd)
    rorder = np.argsort(rev)
    assert (fwd[order] == rev[rorder]).all(), "not symmetric"
    assert (np.asarray(g.adjwgt)[order] == np.asarray(g.adjwgt)[rorder]).all(), "asymmetric weight"
    if sorted_rows:
        for v in range(g.n):
            row = adj[xadj[v]:xadj[v + 1]]
            assert (np.diff(row) > 0).all()


def brute_force_opt(g, k, Lmax):
    """Optimal cut over all k^n assignments with every block <= Lmax (n <= ~16)."""
    n = g.n
    rows = row_index(g)
    adj = np.asarray(g.adjncy)
    w = np.asarray(g.adjwgt, dtype=np.int64)
    vw = np.asarray(g.vwgt, dtype=np.int64)
    best = None
    # enumerate assignments in chunks as base-k digits
    total = k ** n
    chunk = 1 << 16
    powers = k ** np.arange(n, dtype=np.int64)
    for start in range(0, total, chunk):
        ids = np.arange(start, min(total, start + chunk), dtype=np.int64)
        blk = (ids[:, None] // powers[None, :]) % k          # [B, n]
        loads = np.stack([(vw[None, :] * (blk == b)).sum(1) for b in range(k)], 1)
        ok = (loads <= Lmax).all(1)
        if not ok.any():
            continue
        b2 = blk[ok]
        cuts = (w[None, :] * (b2[:, rows] != b2[:, adj])).sum(1) // 2
        c = int(cuts.min())
        best = c if best is None else min(best, c)
    return best
