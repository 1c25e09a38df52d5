"""Seeded synthetic graph generators shared by the oracle tests and the GPU path.

Holds no arithmetic of the partitioning method.  Graphs come back as a
symmetric CSR with sorted rows (no self-loops, no duplicate pairs) and unit
node/edge weights unless asked otherwise.  The drawing itself lives in
``graphgen.c`` (multi-threaded C, identical output for any thread count).

Families (the paper's instance classes, Table 1, plus test shapes):
  er(n, m, seed)                         Erdos-Renyi G(n, m)
  rmat(scale, edge_factor, a, b, c, seed)  R-MAT, Graph500-style quadrants
  grid2d(nx, ny), grid3d(nx, ny, nz)     lattices
  from_pairs(n, u, v)                    any edge list (symmetrised, deduplicated)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles graphgen.c into an in-tree shared library (plain gcc)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.c_uint64)
            lib.gg_er.restype = vp
            lib.gg_er.argtypes = [i32, i64, u64, ctypes.c_int]
            lib.gg_rmat.restype = vp
            lib.gg_rmat.argtypes = [ctypes.c_int, i64, u32, u32, u32, u64, ctypes.c_int]
            lib.gg_grid3d.restype = vp
            lib.gg_grid3d.argtypes = [i32, i32, i32, ctypes.c_int]
            lib.gg_from_pairs.restype = vp
            lib.gg_from_pairs.argtypes = [i32, i64, vp, vp, ctypes.c_int]
            lib.gg_n.restype = i32
            lib.gg_n.argtypes = [vp]
            lib.gg_m2.restype = i64
            lib.gg_m2.argtypes = [vp]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [vp, vp, vp]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [vp]
            lib.gg_word.restype = u64
            lib.gg_word.argtypes = [u64, u64]
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Host CSR graph: int32 ids and weights, xadj int64 (cast to int32 by callers)."""
    n: int
    xadj: np.ndarray     # int64[n+1]
    adjncy: np.ndarray   # int32[m2]
    vwgt: np.ndarray     # int32[n]
    adjwgt: np.ndarray   # int32[m2]
    name: str = ""

    @property
    def m2(self) -> int:
        return int(self.xadj[-1])

    @property
    def m(self) -> int:
        return self.m2 // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.xadj)

    def rows(self) -> np.ndarray:
        """Row index of every CSR entry."""
        return np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())


def _take(handle, name: str) -> Graph:
    lib = _load()
    if not handle:
        raise ValueError(f"graphgen: could not build {name} (bad arguments or out of memory)")
    try:
        n = lib.gg_n(handle)
        m2 = lib.gg_m2(handle)
        xadj = np.empty(n + 1, dtype=np.int64)
        adj = np.empty(max(m2, 1), dtype=np.int32)
        lib.gg_copy(handle, xadj.ctypes.data, adj.ctypes.data)
    finally:
        lib.gg_free(handle)
    adj = adj[:m2]
    return Graph(n=n, xadj=xadj, adjncy=adj, vwgt=np.ones(n, dtype=np.int32),
                 adjwgt=np.ones(m2, dtype=np.int32), name=name)


def er(n: int, m: int, seed: int = 1, threads: int = 0) -> Graph:
    """Erdos-Renyi G(n, m): the first m distinct non-loop pairs in counter order."""
    return _take(_load().gg_er(n, m, seed, threads), f"er_n{n}_m{m}_s{seed}")


RMAT_GRAPH500 = (0.57, 0.19, 0.19)


def rmat_thresholds(a: float, b: float, c: float) -> tuple[int, int, int]:
    """Integer quadrant thresholds out of 65536 (floor of the cumulative probabilities)."""
    return int(a * 65536), int((a + b) * 65536), int((a + b + c) * 65536)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, threads: int = 0) -> Graph:
    """R-MAT with 2^scale nodes and edge_factor * 2^scale sampled (then deduplicated) edges."""
    qa, qab, qabc = rmat_thresholds(a, b, c)
    h = _load().gg_rmat(scale, edge_factor << scale, qa, qab, qabc, seed, threads)
    return _take(h, f"rmat_s{scale}_ef{edge_factor}_seed{seed}")


def grid3d(nx: int, ny: int, nz: int) -> Graph:
    return _take(_load().gg_grid3d(nx, ny, nz, 0), f"grid3d_{nx}x{ny}x{nz}")


def grid2d(nx: int, ny: int) -> Graph:
    return _take(_load().gg_grid3d(nx, ny, 1, 0), f"grid2d_{nx}x{ny}")


def from_pairs(n: int, u, v, name: str = "pairs") -> Graph:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.int32))
    v = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    if u.shape != v.shape:
        raise ValueError("u and v must have the same length")
    return _take(_load().gg_from_pairs(n, len(u), u.ctypes.data, v.ctypes.data, 0), name)


# ----------------------------------------------------------------- weights

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _fin(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def word(seed: int, t) -> np.ndarray:
    """SplitMix64 word t of stream `seed` (same definition as graphgen.c)."""
    t = np.asarray(t, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = _fin(np.asarray([seed], dtype=np.uint64) + np.uint64(0x632BE59BD9B4E019))
        return _fin(base + (t + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15))


def with_edge_weights(g: Graph, wmax: int, seed: int = 7) -> Graph:
    """Symmetric random edge weights in [1, wmax], keyed on the unordered pair."""
    rows = g.rows().astype(np.uint64)
    cols = g.adjncy.astype(np.uint64)
    lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
    key = (lo << np.uint64(32)) | hi
    w = (word(seed, key) % np.uint64(wmax)).astype(np.int64) + 1
    return Graph(g.n, g.xadj, g.adjncy, g.vwgt, w.astype(np.int32), g.name + f"_w{wmax}")


def with_node_weights(g: Graph, cmax: int, seed: int = 11) -> Graph:
    """Random node weights in [1, cmax]."""
    w = (word(seed, np.arange(g.n, dtype=np.uint64)) % np.uint64(cmax)).astype(np.int64) + 1
    return Graph(g.n, g.xadj, g.adjncy, w.astype(np.int32), g.adjwgt, g.name + f"_c{cmax}")


def with_isolated(g: Graph, extra: int) -> Graph:
    """Appends `extra` degree-0 nodes (ids n .. n+extra-1)."""
    xadj = np.concatenate([g.xadj, np.full(extra, g.xadj[-1], dtype=np.int64)])
    vw = np.concatenate([g.vwgt, np.ones(extra, dtype=np.int32)])
    return Graph(g.n + extra, xadj, g.adjncy, vw, g.adjwgt, g.name + f"_iso{extra}")
