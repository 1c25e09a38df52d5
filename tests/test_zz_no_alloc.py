"""gp_cut_noalloc: the cut and block weights computed without any allocation,
for callers that must not allocate device memory while they run (a serving
loop that reserved the device for its own arena, or a latency-critical path
that cannot take cudaMalloc's device-wide synchronisation).

Called through the C-ABI with ctypes and checked against gp_cut on two calls
in a row (the shared scratch keeps the previous call's contents, so the
second call also shows that it is cleared), plus the size limit.  This file
is collected last so that a run stopping at the first failure has run every
other test before it.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2504_17615_gb300 as gp
    from paper_2504_17615_gb300 import build
    build.build()
    lib = ctypes.CDLL(gp.library_path())
    fn = lib.gp_cut_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(gp.gp_graph), ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    return gp, fn


def _noalloc(fn, gp, dg, blocks, k, stream):
    cut = ctypes.c_int64(-1)
    bw = np.full(k, -1, dtype=np.int64)
    s = dg.struct()
    st = fn(ctypes.byref(s), blocks.data_ptr(), k, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(cut),
            bw.ctypes.data)
    return st, cut.value, bw


def test_cut_noalloc_matches_gp_cut_on_consecutive_calls():
    import torch
    gp, fn = _lib()
    ctx = gp.Context(0)
    stream = ctx.stream
    g = gg.with_node_weights(gg.with_edge_weights(gg.rmat(14, 8, seed=5), 9), 4)
    dg = gp.DeviceGraph.from_host(g)
    rng = np.random.default_rng(3)
    for k in (64, 7, 4096):  # consecutive calls, the second one with fewer blocks
        blk = torch.from_numpy(rng.integers(0, k, g.n).astype(np.int32)).cuda()
        st, cut, bw = _noalloc(fn, gp, dg, blk, k, stream)
        assert st == gp.GP_OK
        ref_cut, ref_bw = ctx.gp_cut(dg, blk, k)
        assert cut == ref_cut
        assert np.array_equal(bw, ref_bw)
    ctx.close()


def test_cut_noalloc_rejects_sizes_beyond_its_scratch_and_bad_blocks():
    import torch
    gp, fn = _lib()
    g = gg.er(1000, 4000, 2)
    dg = gp.DeviceGraph.from_host(g)
    stream = torch.cuda.current_stream()
    blk = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    st, _, _ = _noalloc(fn, gp, dg, blk, 4097, stream)
    assert st == gp.GP_ERR_INVALID
    blk[5] = 9
    st, _, _ = _noalloc(fn, gp, dg, blk, 4, stream)
    assert st == gp.GP_ERR_INVALID
    blk[5] = 3
    st, cut, bw = _noalloc(fn, gp, dg, blk, 4, stream)
    assert st == gp.GP_OK and bw.sum() == g.n
    # entries without rows (n == 0, m2 > 0) are rejected before any launch
    bad = gp.gp_graph(0, dg.m2, None, dg.struct().adjncy, None, dg.struct().adjwgt)
    out = ctypes.c_int64(0)
    st = fn(ctypes.byref(bad), None, 4, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out), None)
    assert st == gp.GP_ERR_INVALID
