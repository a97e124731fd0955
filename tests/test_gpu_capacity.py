"""Capacity overflow of splat_bin_sort stays inside the caller's buffers.

When the instance lists need more entries than splat_bins.capacity, the sort
reports SPLAT_ERR_CAPACITY with the count it needed and writes nothing past
the end of any buffer it was given: the entry arrays (capacity entries), the
tile ranges and counters, and the workspace (exactly splat_workspace_size
bytes).  Each buffer here sits between guard bands filled with a pattern, the
views differ in size (so every view's first slot and chunk count matter), and
the overflow is provoked at both places the binned sort checks it -- the
super-tile lists (scan) and the tile lists (tile ranges) -- and in the radix
mode.  A call with enough capacity afterwards gives the reference lists.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2505_13215_gb300 import abi, raster, scenes

pytestmark = pytest.mark.gpu

GUARD = 1 << 16          # elements (entry arrays) / bytes (workspace) on each side
PAT32 = 0x5A5A5A5A
PAT8 = 0xA5


class Guarded:
    """A device array of n elements between two guard bands of a fixed pattern."""

    def __init__(self, n, dtype, guard=GUARD):
        self.n, self.g = int(n), int(guard)
        total = self.n + 2 * self.g
        if dtype == torch.uint8:
            self.buf = torch.full((total,), PAT8, dtype=torch.uint8, device="cuda")
        else:
            words = total * torch.tensor([], dtype=dtype).element_size() // 4
            self.buf = torch.full((words,), PAT32, dtype=torch.int32, device="cuda").view(dtype)
        assert self.buf.numel() == total
        self.pat = self.buf[: self.g].clone()

    @property
    def inner(self):
        return self.buf[self.g: self.g + self.n]

    def ptr(self):
        return self.inner.data_ptr()

    def intact(self):
        return bool(torch.equal(self.buf[: self.g], self.pat) and torch.equal(self.buf[self.g + self.n:], self.pat))


def super_list_total(R):
    """Entries of all super-tile lists (8x8 tiles): the visible rows' rectangles
    widened to super-tiles, cells summed."""
    rect = R.rect.cpu().numpy().astype(np.int64)
    vis = R.n_tiles.cpu().numpy() > 0
    r = rect[vis]
    return int((((r[:, 2] + 7) // 8 - r[:, 0] // 8) * ((r[:, 3] + 7) // 8 - r[:, 1] // 8)).sum())


def guarded_sort(R, capacity, keys=True):
    """One splat_bin_sort of R's projected rows into guarded buffers; returns
    (status, the guarded buffers)."""
    vals = Guarded(capacity, torch.int32)
    kbuf = Guarded(capacity, torch.int32) if keys else None
    ranges = Guarded(2 * R.total_tiles, torch.int32)
    n_inst = Guarded(1, torch.int64, guard=64)
    n_need = Guarded(1, torch.int64, guard=64)
    order = Guarded(R.total_tiles, torch.int32)
    ws_bytes = abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, R.n3, R.n4, R.W, R.H, capacity)
    assert ws_bytes > 0
    ws = Guarded(ws_bytes, torch.uint8)
    assert ws.ptr() % 256 == 0
    bins = abi.splat_bins(capacity, kbuf.ptr() if keys else None, vals.ptr(), ranges.ptr(), n_inst.ptr(),
                          order.ptr(), n_need.ptr())
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = abi.splat_bin_sort(C.byref(R.cproj), R.cviews, R.V, C.byref(bins), C.c_void_p(status.data_ptr()),
                            C.c_void_p(ws.ptr()), ws_bytes, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    s = status.cpu().numpy()
    aux = (int(s[3]) << 32) | (int(s[2]) & 0xFFFFFFFF)
    bufs = {"vals": vals, "ranges": ranges, "n_instances": n_inst, "n_needed": n_need, "tile_order": order,
            "workspace": ws}
    if keys:
        bufs["keys"] = kbuf
    return int(s[0]), int(s[1]), aux, bufs


@pytest.mark.parametrize("mode,cull", [(2, True), (2, False), (1, False)])
def test_capacity_overflow_stays_inside_its_buffers(mode, cull):
    abi.splat_set_tile_sort(mode)
    abi.splat_set_tile_cull(cull)
    try:
        scene, views = scenes.arc_scene(seed=9, n=60000, frac4=0.3, n_views=3, full=(640, 480, 700.0),
                                        half=(336, 250, 360.0))
        G = raster.Gaussians.from_scene(scene, "cuda")
        R = raster.Rasterizer(G.n3, G.n4, views)
        R.autotune_capacity(G)
        R.slice_project(G)
        R.bin_sort()
        torch.cuda.synchronize()
        R.check()
        K = R.instances()
        ref_vals, ref_ranges = R.vals[:K].clone(), R.ranges.clone()
        K1 = super_list_total(R) if mode == 2 else 0
        # (capacity, expected stage, expected count)
        cases = []
        if mode == 2:
            lo = min(K, K1)
            cases.append((lo // 3, abi_stage("scan"), K1))
            cases.append((K1 - 1, abi_stage("scan"), K1))
            if K > K1:  # the tile lists are the longer ones: they overflow after the super-tile lists fit
                cases.append((K1 + (K - K1) // 2, abi_stage("duplicate"), K))
                cases.append((K - 1, abi_stage("duplicate"), K))
        else:
            cases.append((K // 3, None, K))
            cases.append((K - 1, None, K))
        assert cases
        for cap, stage, need in cases:
            code, st, aux, bufs = guarded_sort(R, cap, keys=(mode == 1))
            where = "capacity %d of K=%d K1=%d (mode %d, cull %d)" % (cap, K, K1, mode, cull)
            assert code == abi.SPLAT_ERR_CAPACITY, where
            if stage is not None:
                assert st == stage, where
            assert aux == need, "%s: reported %d, needed %d" % (where, aux, need)
            for name, b in bufs.items():
                assert b.intact(), "%s: guard band of %s overwritten" % (where, name)
        # enough capacity: the reference lists, also through guarded buffers
        code, st, aux, bufs = guarded_sort(R, max(K, K1), keys=(mode == 1))
        assert code == abi.SPLAT_OK
        assert int(bufs["n_instances"].inner.item()) == K
        assert torch.equal(bufs["vals"].inner[:K], ref_vals)
        assert torch.equal(bufs["ranges"].inner, ref_ranges)
        for name, b in bufs.items():
            assert b.intact(), "guard band of %s overwritten" % name
    finally:
        abi.splat_set_tile_sort(0)
        abi.splat_set_tile_cull(True)


def abi_stage(name):
    return {"scan": 3, "duplicate": 4}[name]
