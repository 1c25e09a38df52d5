"""Failure paths, made on the host: no GPU fault, trap or hang is caused.

* An allocator that refuses its N-th request: the call returns GP_ERR_OOM,
  every buffer it took is handed back, and the same context then computes
  the oracle's partition.
* (The bounded device-side wait that returns GP_ERR_TIMEOUT is covered in
  test_gpu_parity.py.)
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gp():
    import torch
    import paper_2504_17615_gb300 as gpmod
    from paper_2504_17615_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return gpmod


class FailingAllocator:
    """torch's caching allocator behind gp_allocator, refusing the fail_at-th request
    (0: never); counts requests and the blocks it still holds."""

    def __init__(self, gp):
        import torch
        self.torch = torch
        self.calls = 0
        self.fail_at = 0
        self.live = {}
        self.struct = gp.gp_allocator(gp.ALLOC_FN(self._alloc), gp.FREE_FN(self._free), None)

    def _alloc(self, nbytes, user, stream):
        self.calls += 1
        if self.fail_at and self.calls == self.fail_at:
            return None
        try:
            p = self.torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        except Exception:
            return None
        self.live[p] = nbytes
        return p

    def _free(self, ptr, nbytes, user, stream):
        self.live.pop(ptr, None)
        self.torch.cuda.caching_allocator_delete(int(ptr))


def test_allocation_failure_returns_oom_and_the_context_recovers(gp):
    import torch
    g = gg.er(20000, 100000, 5)
    ref = orc.partition(g, 8, 0.03, 3)
    fa = FailingAllocator(gp)
    ctx = gp.Context(0, allocator=fa.struct)
    try:
        dg = gp.DeviceGraph.from_host(g)
        ctx.gp_partition(dg, 8, 0.03, 3)  # a clean run: how many allocations one partition makes
        torch.cuda.synchronize()
        total = fa.calls
        assert total > 10 and not fa.live
        for n in sorted({1, 2, total // 3, total // 2, total - 1}):
            fa.calls, fa.fail_at = 0, n
            with pytest.raises(gp.GpError) as e:
                ctx.gp_partition(dg, 8, 0.03, 3)
            assert e.value.status == gp.GP_ERR_OOM, n
            torch.cuda.synchronize()
            assert not fa.live, f"{len(fa.live)} buffers not handed back after failing request {n}"
        fa.fail_at = 0
        blocks, cut, _ = ctx.gp_partition(dg, 8, 0.03, 3)
        assert cut == ref.cut and np.array_equal(blocks.cpu().numpy(), ref.blocks)
    finally:
        ctx.close()
