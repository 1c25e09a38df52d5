"""CPU oracle of the deterministic linear-time multilevel partitioner.

TEST INFRASTRUCTURE ONLY.  ``gp_oracle.c`` is a plain, slow, single-threaded
C implementation of the method of "Linear-Time Multilevel Graph Partitioning
via Edge Sparsification" (label-propagation coarsening, contraction, edge
sparsification per Alg. 1, recursive-bisection initial partitioning, LP
refinement).  Only tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import it; the GPU library never does, and this module
never touches the GPU library.

All graphs are host numpy arrays: xadj int64[n+1], adjncy/vwgt/adjwgt int32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_HDR = os.path.join(_HERE, "gp_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libgp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, INFEASIBLE, OVERFLOW, NOMEM = 0, 1, 2, 3, 4
TAG_ACT, TAG_TIE, TAG_PRIO, TAG_FAV, TAG_SPARSE, TAG_UNIFORM = 1, 2, 3, 4, 5, 6
TAG_RACT, TAG_RTIE, TAG_RPRIO, TAG_IP = 7, 8, 9, 10


def build(force: bool = False) -> str:
    """Compiles the oracle with plain gcc into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class Config(ctypes.Structure):
    """Method parameters; defaults are the paper's (Sec. 4.3, Sec. 6.1) plus the readings R3/R4."""
    _fields_ = [(name, ctypes.c_int32) for name in (
        "tau_e_num", "tau_e_den", "tau_d_num", "tau_d_den", "rho_num", "rho_den",
        "cluster_factor", "coarsest_factor", "shrink_num", "shrink_den",
        "min_shrink_num", "min_shrink_den", "lp_rounds", "lp_subrounds", "ref_rounds",
        "ip_trials", "sparsifier", "two_hop", "isolated", "max_levels", "dbg_max_subrounds")]

    @classmethod
    def default(cls, **kw) -> "Config":
        c = cls(tau_e_num=1, tau_e_den=2, tau_d_num=1, tau_d_den=2, rho_num=4, rho_den=1,
                cluster_factor=160, coarsest_factor=160, shrink_num=5, shrink_den=2,
                min_shrink_num=21, min_shrink_den=20, lp_rounds=5, lp_subrounds=8,
                ref_rounds=5, ip_trials=8, sparsifier=1, two_hop=1, isolated=1,
                max_levels=64, dbg_max_subrounds=-1)
        for k, v in kw.items():
            setattr(c, k, v)
        return c


class Level(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_next", ctypes.c_int32),
                ("m", ctypes.c_int64), ("m_coarse", ctypes.c_int64), ("m_hat", ctypes.c_int64),
                ("m_next", ctypes.c_int64), ("triggered", ctypes.c_int32),
                ("omega_t", ctypes.c_int32), ("n_greater", ctypes.c_int64),
                ("n_equal", ctypes.c_int64), ("threshold", ctypes.c_uint64),
                ("lp_subrounds", ctypes.c_int32), ("lp_moves", ctypes.c_int64),
                ("clusters_lp", ctypes.c_int64), ("clusters_2hop", ctypes.c_int64),
                ("clusters_final", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("lv", Level * 64), ("U", ctypes.c_int64),
                ("Lmax", ctypes.c_int64), ("W", ctypes.c_int64), ("ip_cut", ctypes.c_int64),
                ("cut", ctypes.c_int64), ("rebalance_moves", ctypes.c_int64),
                ("n_coarsest", ctypes.c_int32)]


class SparseStats(ctypes.Structure):
    _fields_ = [("omega_t", ctypes.c_int64), ("n_greater", ctypes.c_int64),
                ("n_equal", ctypes.c_int64), ("m_in", ctypes.c_int64), ("m_out", ctypes.c_int64),
                ("threshold", ctypes.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            G = [i32, P, P, P, P]  # n, xadj, adjncy, vwgt, adjwgt
            sig = {
                "or_key": (u64, [u64, u32, u32, u32]),
                "or_h32": (u32, [u64, u32, u32]),
                "or_h64": (u64, [u64, u32, u32]),
                "or_modularity": (ctypes.c_int, [i32, P, P, P, P, i32, P]),
                "or_validate": (ctypes.c_int, G + [P]),
                "or_lmax": (i64, [i64, i32, i64]),
                "or_cluster_bound": (i64, [i64, i32, i32]),
                "or_cluster": (ctypes.c_int, G + [i64, i32, u64, P, P, P, P]),
                "or_coarsen": (ctypes.c_int, G + [i64, i32, u64, P, P, P, P]),
                "or_coarsen_traced": (ctypes.c_int, G + [i64, i32, u64, P, P, P, P, P, P, i32]),
                "or_contract": (ctypes.c_int, G + [P, i32, P, P, P, P]),
                "or_sparsify": (ctypes.c_int, G + [i64, i32, u64, i32, P, P, P, P, P]),
                "or_m_hat": (i64, [i64, i64, i64, P]),
                "or_trigger": (ctypes.c_int, [i64, i64, P]),
                "or_initial_partition": (ctypes.c_int, G + [i32, i64, u64, i32, P]),
                "or_rebalance": (i64, G + [i32, i64, P]),
                "or_refine": (ctypes.c_int, G + [i32, i64, i32, u64, P, P, P]),
                "or_cut": (i64, [i32, P, P, P, P]),
                "or_partition": (ctypes.c_int, G + [i32, i64, u64, P, P, P, P]),
                "or_coarsen_only": (ctypes.c_int, G + [i32, u64, P, P]),
                "or_free": (None, [P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


@dataclass
class HostGraph:
    n: int
    xadj: np.ndarray
    adjncy: np.ndarray
    vwgt: np.ndarray
    adjwgt: np.ndarray

    @property
    def m2(self) -> int:
        return int(self.xadj[-1])

    @property
    def m(self) -> int:
        return self.m2 // 2


def _args(g):
    keep = [_c(g.xadj, np.int64), _c(g.adjncy, np.int32), _c(g.vwgt, np.int32),
            _c(g.adjwgt, np.int32)]
    return keep, [g.n] + [p for _, p in keep]


def key(seed: int, tag: int, level: int, rnd: int) -> int:
    return _load().or_key(seed, tag, level, rnd)


def h32(k: int, x: int, y: int) -> int:
    return _load().or_h32(k, x, y)


def validate(g) -> tuple[int, int]:
    keep, a = _args(g)
    W = ctypes.c_int64(0)
    rc = _load().or_validate(*a, ctypes.byref(W))
    return rc, W.value


def lmax(W: int, k: int, eps_ppm: int) -> int:
    return _load().or_lmax(W, k, eps_ppm)


def cluster_bound(W: int, k: int, cluster_factor: int = 160) -> int:
    return _load().or_cluster_bound(W, k, cluster_factor)


def eps_to_ppm(eps: float) -> int:
    """eps as integer parts per million (rounded), the form every step uses."""
    return int(round(eps * 1_000_000))


def cluster(g, U: int, level: int, seed: int, cfg: Config | None = None):
    """Cluster labels after LP, 2-hop and isolated-node clustering: (label, nclusters, Level)."""
    cfg = cfg or Config.default()
    keep, a = _args(g)
    label = np.empty(g.n, dtype=np.int32)
    ncl = ctypes.c_int64(0)
    st = Level()
    rc = _load().or_cluster(*a, U, level, seed, ctypes.byref(cfg), label.ctypes.data,
                            ctypes.byref(ncl), ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"or_cluster failed: {rc}")
    return label, ncl.value, st


def coarsen(g, U: int, level: int, seed: int, cfg: Config | None = None):
    """Dense coarse ids: (cmap, n_coarse, Level)."""
    cfg = cfg or Config.default()
    keep, a = _args(g)
    cmap = np.empty(g.n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    st = Level()
    rc = _load().or_coarsen(*a, U, level, seed, ctypes.byref(cfg), cmap.ctypes.data,
                            ctypes.byref(nc), ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"or_coarsen failed: {rc}")
    return cmap, nc.value, st


def coarsen_traced(g, U: int, level: int, seed: int, cfg: Config | None = None, max_digests: int = 512):
    """or_coarsen plus the cluster labels and the label digest after every LP sub-round:
    (label, cmap, n_coarse, Level, digests)."""
    cfg = cfg or Config.default()
    keep, a = _args(g)
    label = np.empty(g.n, dtype=np.int32)
    cmap = np.empty(g.n, dtype=np.int32)
    nc = ctypes.c_int32(0)
    st = Level()
    dig = np.zeros(max_digests, dtype=np.uint64)
    rc = _load().or_coarsen_traced(*a, U, level, seed, ctypes.byref(cfg), label.ctypes.data,
                                   cmap.ctypes.data, ctypes.byref(nc), ctypes.byref(st),
                                   dig.ctypes.data, max_digests)
    if rc != OK:
        raise RuntimeError(f"or_coarsen_traced failed: {rc}")
    return label, cmap, nc.value, st, dig[:min(st.lp_subrounds, max_digests)]


def label_digest(label) -> int:
    """The digest or_coarsen_traced records: sum of mix(v << 32 | label[v]) mod 2^64."""
    lab = np.asarray(label, dtype=np.int64) & 0xFFFFFFFF
    v = np.arange(len(lab), dtype=np.uint64)
    z = (v << np.uint64(32)) | lab.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
        return int(z.sum(dtype=np.uint64))


def _take_graph(n, px, pa, pv, pw) -> HostGraph:
    lib = _load()
    xadj = np.ctypeslib.as_array(ctypes.cast(px, ctypes.POINTER(ctypes.c_int64)), (n + 1,)).copy()
    m2 = int(xadj[-1])
    adj = np.ctypeslib.as_array(ctypes.cast(pa, ctypes.POINTER(ctypes.c_int32)), (max(m2, 1),))[:m2].copy()
    vw = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_int32)), (max(n, 1),))[:n].copy()
    aw = np.ctypeslib.as_array(ctypes.cast(pw, ctypes.POINTER(ctypes.c_int32)), (max(m2, 1),))[:m2].copy()
    for p in (px, pa, pv, pw):
        lib.or_free(p)
    return HostGraph(n, xadj, adj, vw, aw)


def contract(g, cmap: np.ndarray, n_coarse: int) -> HostGraph:
    keep, a = _args(g)
    cm, pcm = _c(cmap, np.int32)
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    rc = _load().or_contract(*a, pcm, n_coarse, *[ctypes.byref(p) for p in ptrs])
    if rc != OK:
        raise RuntimeError(f"or_contract failed: {rc}")
    return _take_graph(n_coarse, *[p.value for p in ptrs])


def sparsify(g, m_hat: int, level: int, seed: int, mode: int = 1):
    """Returns (sparsified graph, SparseStats)."""
    keep, a = _args(g)
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    st = SparseStats()
    rc = _load().or_sparsify(*a, m_hat, level, seed, mode, *[ctypes.byref(p) for p in ptrs],
                             ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"or_sparsify failed: {rc}")
    return _take_graph(g.n, *[p.value for p in ptrs]), st


def h64(k: int, x: int, y: int) -> int:
    """All 64 bits of the mix behind h32 (the order of the exact-count sampler)."""
    return _load().or_h64(k, x, y)


@dataclass
class Modularity:
    """Sec. 5 for a clustering, from exact integer totals over the CSR entries."""
    w_internal: int
    w_total: int
    vol_max: int
    vol_sq: int

    @property
    def inside(self) -> float:  # sum_i e_ii
        return self.w_internal / self.w_total

    @property
    def q(self) -> float:  # Q_C
        return self.inside - self.vol_sq / float(self.w_total) ** 2

    @property
    def alpha(self) -> float:  # alpha_C
        return self.vol_max / self.w_total

    @property
    def bound(self) -> float:  # Lemma 2: lower bound of the weight fraction between clusters
        return 1.0 - self.q - self.alpha


def modularity(g, labels, nlabels: int) -> Modularity:
    keep, a = _args(g)
    lab, plab = _c(labels, np.int32)
    out = np.zeros(4, dtype=np.int64)
    rc = _load().or_modularity(g.n, a[1], a[2], a[4], plab, nlabels, out.ctypes.data)
    if rc != OK:
        raise RuntimeError(f"or_modularity failed: {rc}")
    return Modularity(int(out[0]), int(out[1]), int(out[2]), int(np.uint64(out[3])))


def m_hat(m: int, n: int, n_next: int, cfg: Config | None = None) -> int:
    cfg = cfg or Config.default()
    return _load().or_m_hat(m, n, n_next, ctypes.byref(cfg))


def trigger(m_coarse: int, mh: int, cfg: Config | None = None) -> bool:
    cfg = cfg or Config.default()
    return bool(_load().or_trigger(m_coarse, mh, ctypes.byref(cfg)))


def initial_partition(g, k: int, eps_ppm: int, seed: int, trials: int = 8) -> np.ndarray:
    keep, a = _args(g)
    blk = np.empty(g.n, dtype=np.int32)
    rc = _load().or_initial_partition(*a, k, eps_ppm, seed, trials, blk.ctypes.data)
    if rc != OK:
        raise RuntimeError(f"or_initial_partition failed: {rc}")
    return blk


def rebalance(g, k: int, Lmax: int, blk: np.ndarray) -> tuple[np.ndarray, int]:
    keep, a = _args(g)
    b = np.array(blk, dtype=np.int32, copy=True)
    moves = _load().or_rebalance(*a, k, Lmax, b.ctypes.data)
    return b, moves


def refine(g, k: int, Lmax: int, level: int, seed: int, blk: np.ndarray,
           cfg: Config | None = None) -> tuple[np.ndarray, int]:
    cfg = cfg or Config.default()
    keep, a = _args(g)
    b = np.array(blk, dtype=np.int32, copy=True)
    mv = ctypes.c_int64(0)
    rc = _load().or_refine(*a, k, Lmax, level, seed, ctypes.byref(cfg), b.ctypes.data,
                           ctypes.byref(mv))
    if rc != OK:
        raise RuntimeError(f"or_refine failed: {rc}")
    return b, mv.value


def cut(g, blk: np.ndarray) -> int:
    keep, a = _args(g)
    b, pb = _c(blk, np.int32)
    return _load().or_cut(g.n, a[1], a[2], a[4], pb)


@dataclass
class Result:
    rc: int
    blocks: np.ndarray
    cut: int
    stats: Stats = field(repr=False)

    def levels(self) -> list[dict]:
        return [self.stats.lv[i].as_dict() for i in range(self.stats.levels)]


def coarsen_only(g, k: int, seed: int, cfg: Config | None = None) -> Stats:
    """Runs only the coarsening phase (Alg. 1) and returns its per-level records."""
    cfg = cfg or Config.default()
    keep, a = _args(g)
    st = Stats()
    rc = _load().or_coarsen_only(*a, k, seed, ctypes.byref(cfg), ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"or_coarsen_only failed: {rc}")
    return st


def partition(g, k: int, eps: float, seed: int, cfg: Config | None = None) -> Result:
    cfg = cfg or Config.default()
    keep, a = _args(g)
    blk = np.zeros(g.n, dtype=np.int32)
    c = ctypes.c_int64(0)
    st = Stats()
    rc = _load().or_partition(*a, k, eps_to_ppm(eps), seed, ctypes.byref(cfg), blk.ctypes.data,
                              ctypes.byref(c), ctypes.byref(st))
    return Result(rc, blk, c.value, st)
