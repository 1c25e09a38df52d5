"""Python binding of the GB300 multilevel graph partitioner (include/gp.h).

Argument marshalling only: every step runs in the CUDA library
``_build/libgp_gb300.so`` (built from ``csrc/`` for sm_103a).  PyTorch
provides device memory (through the library's allocator hook) and streams.
There is no CPU fallback: without the compiled library or a GPU every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

GP_OK, GP_ERR_INVALID, GP_ERR_INFEASIBLE, GP_ERR_OVERFLOW = 0, 1, 2, 3
GP_ERR_OOM, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_BUDGET = 4, 5, 6, 7
GP_SPARSIFY_NONE, GP_SPARSIFY_TWEIGHT, GP_SPARSIFY_UNIFORM, GP_SPARSIFY_TWEIGHT_EXACT = 0, 1, 2, 3
STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_INVALID", 2: "GP_ERR_INFEASIBLE", 3: "GP_ERR_OVERFLOW",
                4: "GP_ERR_OOM", 5: "GP_ERR_CUDA", 6: "GP_ERR_TIMEOUT", 7: "GP_ERR_BUDGET"}


class GpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ------------------------------------------------------------------ structs

class gp_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m2", ctypes.c_int64), ("xadj", ctypes.c_void_p),
                ("adjncy", ctypes.c_void_p), ("vwgt", ctypes.c_void_p), ("adjwgt", ctypes.c_void_p)]


class gp_batch_item(ctypes.Structure):
    _fields_ = [("g", gp_graph), ("k", ctypes.c_int32), ("eps", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("blocks", ctypes.c_void_p), ("cut", ctypes.c_int64), ("status", ctypes.c_int),
                ("engine", ctypes.c_int32), ("stats", ctypes.c_void_p)]


GP_TUNE_CLASSES = 12


class gp_batch_tuning(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int32), ("threads", ctypes.c_int32), ("max_entries", ctypes.c_int64),
                ("max_nodes", ctypes.c_int64), ("arena_cap_bytes", ctypes.c_int64),
                ("arena_bytes", ctypes.c_int64), ("classes", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("class_entries", ctypes.c_int64 * GP_TUNE_CLASSES),
                ("class_items", ctypes.c_int32 * GP_TUNE_CLASSES),
                ("class_threads", ctypes.c_int32 * GP_TUNE_CLASSES),
                ("class_engine_gps", ctypes.c_double * GP_TUNE_CLASSES),
                ("class_path_gps", ctypes.c_double * GP_TUNE_CLASSES), ("tune_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f in ("engine", "threads", "max_entries", "max_nodes", "arena_cap_bytes",
                                           "arena_bytes", "classes", "tune_ms")}
        d["class_table"] = [{"max_entries": self.class_entries[i], "items": self.class_items[i],
                             "engine_threads": self.class_threads[i],
                             "engine_graphs_per_s": self.class_engine_gps[i],
                             "path_graphs_per_s": self.class_path_gps[i]}
                            for i in range(self.classes) if self.class_items[i] > 0]
        return d


class gp_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m2", ctypes.c_int64), ("xadj", ctypes.c_void_p),
                ("adjncy", ctypes.c_void_p), ("vwgt", ctypes.c_void_p), ("adjwgt", ctypes.c_void_p),
                ("k", ctypes.c_int32), ("eps", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("blocks", ctypes.c_void_p)]


class gp_response(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cut", ctypes.c_int64), ("queued_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("start_order", ctypes.c_int64),
                ("estimate_bytes", ctypes.c_int64), ("peak_reserved_bytes", ctypes.c_int64),
                ("peak_used_bytes", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class gp_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


_CFG_FIELDS = ("tau_e_num", "tau_e_den", "tau_d_num", "tau_d_den", "rho_num", "rho_den",
               "cluster_factor", "coarsest_factor", "shrink_num", "shrink_den",
               "min_shrink_num", "min_shrink_den", "lp_rounds", "lp_subrounds", "ref_rounds",
               "ip_trials", "sparsifier", "two_hop", "isolated", "max_levels",
               "dbg_max_subrounds", "validate", "small_lp_nodes")


class gp_config(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in _CFG_FIELDS]


class gp_level_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_next", ctypes.c_int32), ("m", ctypes.c_int64),
                ("m_coarse", ctypes.c_int64), ("m_hat", ctypes.c_int64), ("m_next", ctypes.c_int64),
                ("triggered", ctypes.c_int32), ("omega_t", ctypes.c_int32),
                ("n_greater", ctypes.c_int64), ("n_equal", ctypes.c_int64),
                ("threshold", ctypes.c_uint64), ("lp_subrounds", ctypes.c_int32),
                ("lp_moves", ctypes.c_int64), ("clusters_lp", ctypes.c_int64),
                ("clusters_2hop", ctypes.c_int64), ("clusters_final", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class gp_modularity_stats(ctypes.Structure):
    _fields_ = [("w_internal", ctypes.c_int64), ("w_total", ctypes.c_int64), ("vol_max", ctypes.c_int64),
                ("vol_sq", ctypes.c_uint64), ("inside", ctypes.c_double), ("q", ctypes.c_double),
                ("alpha", ctypes.c_double), ("bound", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class gp_partition_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("lv", gp_level_stats * 64), ("U", ctypes.c_int64),
                ("Lmax", ctypes.c_int64), ("W", ctypes.c_int64), ("ip_cut", ctypes.c_int64),
                ("cut", ctypes.c_int64), ("rebalance_moves", ctypes.c_int64),
                ("n_coarsest", ctypes.c_int32), ("ms_coarsen", ctypes.c_double),
                ("ms_initial", ctypes.c_double), ("ms_uncoarsen", ctypes.c_double),
                ("ms_total", ctypes.c_double)]

    def levels_list(self) -> list[dict]:
        return [self.lv[i].as_dict() for i in range(self.levels)]


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libgp_gb300.so")


def _load():
    """Loads the compiled library (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, i32, i64, u64, d = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                               ctypes.c_double)
        G = ctypes.POINTER(gp_graph)
        C = ctypes.POINTER(gp_config)
        S = ctypes.POINTER(gp_level_stats)
        sig = {
            "gp_config_default": (None, [C]),
            "gp_version": (ctypes.c_char_p, []),
            "gp_launch_count": (i64, []),
            "gp_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P, ctypes.POINTER(gp_allocator)]),
            "gp_destroy": (None, [P]),
            "gp_set_wait_limit": (None, [P, i64]),
            "gp_last_error": (ctypes.c_char_p, [P]),
            "gp_coarsen": (ctypes.c_int, [P, G, i64, i32, u64, C, P, P, ctypes.POINTER(i32), S]),
            "gp_contract": (ctypes.c_int, [P, G, P, i32, G]),
            "gp_sparsify": (ctypes.c_int, [P, G, i64, i32, u64, i32, G, S]),
            "gp_partition": (ctypes.c_int, [P, G, i32, d, u64, C, P, ctypes.POINTER(i64),
                                            ctypes.POINTER(gp_partition_stats)]),
            "gp_partition_host": (ctypes.c_int, [P, i32, i64, P, P, P, P, i32, d, u64, C, P,
                                                 ctypes.POINTER(i64), ctypes.POINTER(gp_partition_stats)]),
            "gp_initial_partition": (ctypes.c_int, [P, G, i32, d, u64, C, P]),
            "gp_rebalance": (ctypes.c_int, [P, G, i32, i64, P, ctypes.POINTER(i64)]),
            "gp_refine": (ctypes.c_int, [P, G, i32, i64, i32, u64, C, P, ctypes.POINTER(i64)]),
            "gp_project": (ctypes.c_int, [P, i32, P, P, P]),
            "gp_cut": (ctypes.c_int, [P, G, P, i32, ctypes.POINTER(i64), P]),
            "gp_graph_release": (None, [P, G]),
            "gp_profile_enable": (None, [P, ctypes.c_int]),
            "gp_profile_reset": (None, [P]),
            "gp_profile_count": (ctypes.c_int, []),
            "gp_profile_name": (ctypes.c_char_p, [ctypes.c_int]),
            "gp_profile_read": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(d),
                                               ctypes.POINTER(d)]),
            "gp_measure_random_reads": (ctypes.c_int, [P, i64, i64, ctypes.POINTER(d)]),
            "gp_partition_batch": (ctypes.c_int, [P, ctypes.POINTER(gp_batch_item), i32, i32, C]),
            "gp_batch_tuning_default": (None, [ctypes.POINTER(gp_batch_tuning)]),
            "gp_batch_set_tuning": (ctypes.c_int, [P, ctypes.POINTER(gp_batch_tuning)]),
            "gp_batch_get_tuning": (ctypes.c_int, [P, ctypes.POINTER(gp_batch_tuning)]),
            "gp_batch_autotune": (ctypes.c_int, [P, ctypes.POINTER(gp_batch_item), i32, i32, C,
                                                 ctypes.POINTER(gp_batch_tuning)]),
            "gp_server_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, i32, i64, C]),
            "gp_server_submit": (ctypes.c_int, [P, ctypes.POINTER(gp_request), ctypes.POINTER(i64)]),
            "gp_server_wait": (ctypes.c_int, [P, i64, ctypes.POINTER(gp_response)]),
            "gp_server_destroy": (None, [P]),
            "gp_server_set_max_bypass": (None, [P, i32]),
            "gp_modularity": (ctypes.c_int, [P, ctypes.POINTER(gp_graph), P, i32, ctypes.POINTER(gp_modularity_stats)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def default_config(**kw) -> gp_config:
    c = gp_config()
    _load().gp_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


# --------------------------------------------------------------- graphs

@dataclass
class DeviceGraph:
    """A CSR graph in device memory (torch int32 tensors)."""
    n: int
    m2: int
    xadj: "object"
    adjncy: "object"
    vwgt: "object"
    adjwgt: "object"

    def struct(self) -> gp_graph:
        return gp_graph(self.n, self.m2, self.xadj.data_ptr(), self.adjncy.data_ptr(),
                        self.vwgt.data_ptr(), self.adjwgt.data_ptr())

    @staticmethod
    def from_host(g, device="cuda") -> "DeviceGraph":
        import torch
        xadj = np.asarray(g.xadj)
        if int(xadj[-1]) >= 2**31:
            raise ValueError("graph too large for int32 offsets")
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(device)
        adj = g.adjncy if len(g.adjncy) else np.zeros(1, np.int32)
        aw = g.adjwgt if len(g.adjwgt) else np.zeros(1, np.int32)
        vw = g.vwgt if len(g.vwgt) else np.zeros(1, np.int32)
        return DeviceGraph(int(g.n), int(xadj[-1]), t(xadj), t(adj), t(vw), t(aw))

    def to_host(self):
        return HostCopy(self.n, self.xadj.cpu().numpy().astype(np.int64),
                        self.adjncy.cpu().numpy()[:self.m2], self.vwgt.cpu().numpy()[:self.n],
                        self.adjwgt.cpu().numpy()[:self.m2])


@dataclass
class HostCopy:
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


def _device_view(ptr: int, count: int):
    """Non-owning torch int32 view of library-owned device memory."""
    import torch

    class _Iface:
        pass

    o = _Iface()
    o.__cuda_array_interface__ = {"shape": (max(count, 0),), "typestr": "<i4",
                                  "data": (int(ptr) if count > 0 else 0, False), "version": 3}
    if count == 0:
        return torch.zeros(0, dtype=torch.int32, device="cuda")
    return torch.as_tensor(o, device="cuda")


class LibGraph:
    """A graph allocated by the library (gp_contract / gp_sparsify)."""

    def __init__(self, ctx: "Context", g: gp_graph):
        self.ctx = ctx
        self.g = g

    @property
    def n(self) -> int:
        return self.g.n

    @property
    def m2(self) -> int:
        return self.g.m2

    def struct(self) -> gp_graph:
        return self.g

    def tensors(self):
        return (_device_view(self.g.xadj, self.g.n + 1), _device_view(self.g.adjncy, self.g.m2),
                _device_view(self.g.vwgt, self.g.n), _device_view(self.g.adjwgt, self.g.m2))

    def to_host(self) -> HostCopy:
        x, a, v, w = (t.cpu().numpy() for t in self.tensors())
        return HostCopy(self.g.n, x.astype(np.int64), a, v, w)

    def release(self):
        if self.g is not None and self.ctx is not None and self.ctx.ptr:
            self.ctx.lib.gp_graph_release(self.ctx.ptr, ctypes.byref(self.g))
        self.g = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


# -------------------------------------------------------------- context

class Context:
    """A library context on one device and stream.  Device memory comes from the
    library's own stream-ordered pool, or from torch's caching allocator when
    use_torch_allocator is set (one Python call per allocation: slower)."""

    def __init__(self, device: int = 0, stream=None, use_torch_allocator: bool = False,
                 allocator: "gp_allocator | None" = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device available: the partitioner runs on the GPU only")
        self.lib = _load()
        self.device = device
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._keep = []
        alloc = None
        if use_torch_allocator:
            dev = device

            def _alloc(nbytes, user, stream):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
                except Exception:
                    return None

            def _free(ptr, nbytes, user, stream):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            alloc = gp_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
            self._keep.append(alloc)
        if allocator is not None:  # a caller's gp_allocator (its callbacks must outlive the context)
            alloc = allocator
            self._keep.append(alloc)
        p = ctypes.c_void_p()
        st = self.lib.gp_create(ctypes.byref(p), device, ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(alloc) if alloc is not None else None)
        if st != GP_OK:
            raise GpError(st, "gp_create failed")
        self.ptr = p.value

    def close(self):
        if getattr(self, "ptr", None):
            self.lib.gp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != GP_OK:
            raise GpError(st, (self.lib.gp_last_error(self.ptr) or b"").decode())

    # --- the C-ABI calls, same names ---

    def gp_set_wait_limit(self, spins: int):
        """Iteration limit of device-side waits (0: default, < 0: give up at once)."""
        self.lib.gp_set_wait_limit(self.ptr, int(spins))

    def gp_coarsen(self, g, U: int, level: int, seed: int, cfg: gp_config | None = None,
                   want_label: bool = False):
        """Returns (cmap tensor, n_coarse, gp_level_stats[, label tensor])."""
        torch = self.torch
        cmap = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
        label = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda") if want_label else None
        nc = ctypes.c_int32(0)
        st = gp_level_stats()
        s = g.struct()
        self._check(self.lib.gp_coarsen(self.ptr, ctypes.byref(s), U, level, seed,
                                        ctypes.byref(cfg) if cfg is not None else None,
                                        cmap.data_ptr(), label.data_ptr() if label is not None else None,
                                        ctypes.byref(nc), ctypes.byref(st)))
        if want_label:
            return cmap[:g.n], nc.value, st, label[:g.n]
        return cmap[:g.n], nc.value, st

    def gp_contract(self, g, cmap, n_coarse: int) -> LibGraph:
        out = gp_graph()
        s = g.struct()
        self._check(self.lib.gp_contract(self.ptr, ctypes.byref(s), cmap.data_ptr(), n_coarse,
                                         ctypes.byref(out)))
        return LibGraph(self, out)

    def gp_sparsify(self, g, m_hat: int, level: int, seed: int, mode: int = GP_SPARSIFY_TWEIGHT):
        out = gp_graph()
        st = gp_level_stats()
        s = g.struct()
        self._check(self.lib.gp_sparsify(self.ptr, ctypes.byref(s), m_hat, level, seed, mode,
                                         ctypes.byref(out), ctypes.byref(st)))
        return LibGraph(self, out), st

    def gp_partition(self, g, k: int, eps: float, seed: int, cfg: gp_config | None = None,
                     blocks=None):
        """Returns (blocks tensor, cut, gp_partition_stats)."""
        torch = self.torch
        if blocks is None:
            blocks = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
        cut = ctypes.c_int64(0)
        st = gp_partition_stats()
        s = g.struct()
        self._check(self.lib.gp_partition(self.ptr, ctypes.byref(s), k, eps, seed,
                                          ctypes.byref(cfg) if cfg is not None else None,
                                          blocks.data_ptr(), ctypes.byref(cut), ctypes.byref(st)))
        return blocks[:g.n], cut.value, st

    def _batch_items(self, jobs, with_stats=False):
        torch = self.torch
        arr = (gp_batch_item * max(len(jobs), 1))()
        outs, stats = [], []
        for i, (g, k, eps, seed) in enumerate(jobs):
            b = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
            outs.append(b)
            arr[i].g = g.struct()
            arr[i].k, arr[i].eps, arr[i].seed = k, eps, seed
            arr[i].blocks = b.data_ptr()
            if with_stats:
                st = gp_partition_stats()
                stats.append(st)
                arr[i].stats = ctypes.addressof(st)
        return arr, outs, stats

    def gp_partition_batch(self, jobs, workers: int = 8, cfg: gp_config | None = None, check: bool = True,
                           details: bool = False):
        """jobs: list of (graph, k, eps, seed).  Returns [(blocks tensor, cut)] in job order
        ([(blocks, cut, status)] without raising when check is False; with details, every tuple
        also carries the item's engine flag and its gp_partition_stats)."""
        arr, outs, stats = self._batch_items(jobs, with_stats=details)
        st = self.lib.gp_partition_batch(self.ptr, arr, len(jobs), workers,
                                         ctypes.byref(cfg) if cfg is not None else None)
        if check:
            self._check(st)
        res = []
        for i in range(len(jobs)):
            r = (outs[i][:jobs[i][0].n], arr[i].cut) + (() if check else (arr[i].status,))
            if details:
                r = r + (arr[i].engine, stats[i])
            res.append(r)
        return res

    def batch_tuning(self) -> gp_batch_tuning:
        t = gp_batch_tuning()
        self._check(self.lib.gp_batch_get_tuning(self.ptr, ctypes.byref(t)))
        return t

    def batch_set_tuning(self, **kw) -> gp_batch_tuning:
        """Engine settings; fields not given keep their defaults (gp_batch_tuning_default)."""
        t = gp_batch_tuning()
        self.lib.gp_batch_tuning_default(ctypes.byref(t))
        for k, v in kw.items():
            setattr(t, k, v)
        self._check(self.lib.gp_batch_set_tuning(self.ptr, ctypes.byref(t)))
        return t

    def batch_autotune(self, jobs, workers: int = 8, cfg: gp_config | None = None) -> gp_batch_tuning:
        arr, outs, _ = self._batch_items(jobs)
        t = gp_batch_tuning()
        self._check(self.lib.gp_batch_autotune(self.ptr, arr, len(jobs), workers,
                                               ctypes.byref(cfg) if cfg is not None else None,
                                               ctypes.byref(t)))
        return t

    def gp_partition_host(self, n: int, m2: int, xadj, adjncy, vwgt, adjwgt, k: int, eps: float,
                          seed: int, cfg: gp_config | None = None, blocks=None):
        """Host arrays in (numpy or pinned torch CPU tensors), host block ids out."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        if blocks is None:
            blocks = np.empty(max(n, 1), dtype=np.int32)
        cut = ctypes.c_int64(0)
        st = gp_partition_stats()
        self._check(self.lib.gp_partition_host(self.ptr, n, m2, ptr(xadj), ptr(adjncy), ptr(vwgt),
                                               ptr(adjwgt), k, eps, seed,
                                               ctypes.byref(cfg) if cfg is not None else None,
                                               ptr(blocks), ctypes.byref(cut), ctypes.byref(st)))
        return blocks, cut.value, st

    def gp_initial_partition(self, g, k: int, eps: float, seed: int, cfg: gp_config | None = None):
        torch = self.torch
        blocks = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
        s = g.struct()
        self._check(self.lib.gp_initial_partition(self.ptr, ctypes.byref(s), k, eps, seed,
                                                  ctypes.byref(cfg) if cfg is not None else None,
                                                  blocks.data_ptr()))
        return blocks[:g.n]

    def gp_rebalance(self, g, k: int, Lmax: int, blocks) -> int:
        mv = ctypes.c_int64(0)
        s = g.struct()
        self._check(self.lib.gp_rebalance(self.ptr, ctypes.byref(s), k, Lmax, blocks.data_ptr(),
                                          ctypes.byref(mv)))
        return mv.value

    def gp_refine(self, g, k: int, Lmax: int, level: int, seed: int, blocks,
                  cfg: gp_config | None = None) -> int:
        mv = ctypes.c_int64(0)
        s = g.struct()
        self._check(self.lib.gp_refine(self.ptr, ctypes.byref(s), k, Lmax, level, seed,
                                       ctypes.byref(cfg) if cfg is not None else None,
                                       blocks.data_ptr(), ctypes.byref(mv)))
        return mv.value

    def gp_project(self, cmap, coarse, n: int):
        fine = self.torch.empty(max(n, 1), dtype=self.torch.int32, device="cuda")
        self._check(self.lib.gp_project(self.ptr, n, cmap.data_ptr(), coarse.data_ptr(), fine.data_ptr()))
        return fine[:n]

    def gp_cut(self, g, blocks, k: int):
        cut = ctypes.c_int64(0)
        bw = np.zeros(k, dtype=np.int64)
        s = g.struct()
        self._check(self.lib.gp_cut(self.ptr, ctypes.byref(s), blocks.data_ptr(), k, ctypes.byref(cut),
                                    bw.ctypes.data))
        return cut.value, bw

    # --- profiling ---

    def profile(self, on: bool = True):
        self.lib.gp_profile_enable(self.ptr, 1 if on else 0)

    def profile_reset(self):
        self.lib.gp_profile_reset(self.ptr)

    def profile_read(self) -> dict:
        out = {}
        for i in range(self.lib.gp_profile_count()):
            la, ms, by = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
            self._check(self.lib.gp_profile_read(self.ptr, i, ctypes.byref(la), ctypes.byref(ms),
                                                 ctypes.byref(by)))
            out[self.lib.gp_profile_name(i).decode()] = {"launches": la.value, "ms": ms.value,
                                                         "bytes": by.value}
        return out

    def gp_modularity(self, g, labels, nlabels: int) -> gp_modularity_stats:
        """Sec. 5 modularity of a clustering given as device labels in [0, nlabels)."""
        st = gp_modularity_stats()
        s = g.struct()
        self._check(self.lib.gp_modularity(self.ptr, ctypes.byref(s), ctypes.c_void_p(labels.data_ptr()),
                                           nlabels, ctypes.byref(st)))
        return st

    def measure_random_reads(self, array_bytes: int, reads: int) -> float:
        """Random 4-byte reads per second from an array of array_bytes bytes."""
        r = ctypes.c_double(0)
        self._check(self.lib.gp_measure_random_reads(self.ptr, array_bytes, reads, ctypes.byref(r)))
        return r.value


def version() -> str:
    return _load().gp_version().decode()


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_load().gp_launch_count())


class Server:
    """The library's request loop (gp_server_*): requests from host arrays, answered by worker
    threads with their own streams, admitted against a device-memory budget."""

    def __init__(self, device: int = 0, workers: int = 8, hbm_budget: int = 96 << 30,
                 cfg: gp_config | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device available: the partitioner runs on the GPU only")
        self.lib = _load()
        p = ctypes.c_void_p()
        st = self.lib.gp_server_create(ctypes.byref(p), device, workers, hbm_budget,
                                       ctypes.byref(cfg) if cfg is not None else None)
        if st != GP_OK:
            raise GpError(st, "gp_server_create failed")
        self.ptr = p.value
        self._live = {}

    def set_max_bypass(self, max_bypass: int):
        """At most this many younger requests may start ahead of the oldest queued one."""
        self.lib.gp_server_set_max_bypass(self.ptr, int(max_bypass))

    def submit(self, g, k: int, eps: float, seed: int) -> int:
        """g: a host graph (numpy CSR with int32 ids and weights).  Returns a ticket."""
        arrs = [np.ascontiguousarray(g.xadj, dtype=np.int32), np.ascontiguousarray(g.adjncy, dtype=np.int32),
                np.ascontiguousarray(g.vwgt, dtype=np.int32), np.ascontiguousarray(g.adjwgt, dtype=np.int32)]
        blocks = np.empty(max(g.n, 1), dtype=np.int32)
        r = gp_request(g.n, int(arrs[0][-1]) if g.n else 0, *[a.ctypes.data for a in arrs], k, eps, seed,
                       blocks.ctypes.data)
        t = ctypes.c_int64(0)
        st = self.lib.gp_server_submit(self.ptr, ctypes.byref(r), ctypes.byref(t))
        if st != GP_OK:
            raise GpError(st, "gp_server_submit failed")
        self._live[t.value] = (arrs, blocks, g.n)
        return t.value

    def wait(self, ticket: int):
        """Blocks until done.  Returns (blocks, cut, gp_response)."""
        resp = gp_response()
        st = self.lib.gp_server_wait(self.ptr, ticket, ctypes.byref(resp))
        if st != GP_OK:
            raise GpError(st, "gp_server_wait failed")
        _, blocks, n = self._live.pop(ticket)
        return blocks[:n], resp.cut, resp

    def close(self):
        if getattr(self, "ptr", None):
            self.lib.gp_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
