"""splat_bin_sort_noalloc against splat_bin_sort, through the C ABI.

The allocation-free variant is for callers that cannot allocate device memory
when they sort -- a plugin whose host application owns the whole GPU memory
budget, or a frame loop that must not call cudaMalloc / cudaFree because those
can synchronise the device.  It takes its scratch from a fixed array inside the
library instead of a workspace argument.  Its output must equal the regular
entry point's output exactly (integer lists), call after call, since every call
reuses the same array.
"""
import ctypes as C

import pytest
import torch

from paper_2505_13215_gb300 import abi, raster, scenes

pytestmark = pytest.mark.gpu


def _bins(capacity, total_tiles):
    keys = torch.zeros(capacity, dtype=torch.int32, device="cuda")
    vals = torch.zeros(capacity, dtype=torch.int32, device="cuda")
    ranges = torch.zeros(2 * total_tiles, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    c = abi.splat_bins(capacity, keys.data_ptr(), vals.data_ptr(), ranges.data_ptr(), n.data_ptr())
    return c, keys, vals, ranges, n


def _noalloc_sort(R, c, status):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = abi.splat_bin_sort_noalloc(C.byref(R.cproj), R.cviews, R.V, C.byref(c), C.c_void_p(status.data_ptr()), stream)
    assert rc == abi.SPLAT_OK, abi.status_string(rc)
    torch.cuda.synchronize()
    assert int(status[0]) == abi.SPLAT_OK, abi.status_string(int(status[0]))


def _reference_lists(R, G):
    R.autotune_capacity(G)
    R.slice_project(G)
    R.bin_sort()
    torch.cuda.synchronize()
    R.check()
    K = R.instances()
    return K, R.keys[:K].clone(), R.vals[:K].clone(), R.ranges.clone()


def test_noalloc_bin_sort_matches_workspace_version_twice():
    # a larger, different problem first (two 640x480 views of a dense scene, so
    # the saturation head and the tail segments both run): whatever it leaves in
    # the shared scratch must not leak into the calls compared below
    big_scene, base = scenes.video_scene(seed=7, n3=20000, n4=10000, W=640, H=480, f=700.0)
    big_views = scenes.jittered_views(base[0], 2, seed=8)
    Gb = raster.Gaussians.from_scene(big_scene, "cuda")
    Rb = raster.Rasterizer(Gb.n3, Gb.n4, big_views)
    Kb, bkeys, bvals, branges = _reference_lists(Rb, Gb)
    assert abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, Gb.n3, Gb.n4, Rb.W, Rb.H, Rb.capacity) <= \
        abi.SPLAT_NOALLOC_SCRATCH_BYTES
    cb, keys_b, vals_b, ranges_b, n_b = _bins(Rb.capacity, Rb.total_tiles)
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    _noalloc_sort(Rb, cb, status)
    assert int(n_b.item()) == Kb
    assert torch.equal(vals_b[:Kb], bvals) and torch.equal(ranges_b, branges)

    scene, views = scenes.small_scene(seed=0)
    G = raster.Gaussians.from_scene(scene, "cuda")
    R = raster.Rasterizer(G.n3, G.n4, views)
    K, ref_keys, ref_vals, ref_ranges = _reference_lists(R, G)
    c, keys, vals, ranges, n = _bins(R.capacity, R.total_tiles)
    for call in range(2):
        keys.fill_(-1)
        vals.fill_(-1)
        ranges.fill_(-1)
        _noalloc_sort(R, c, status)
        assert int(n.item()) == K
        assert torch.equal(keys[:K], ref_keys), "call %d keys" % call
        assert torch.equal(vals[:K], ref_vals), "call %d vals" % call
        assert torch.equal(ranges, ref_ranges), "call %d ranges" % call


def test_noalloc_rejects_problems_larger_than_its_scratch():
    scene, views = scenes.small_scene(seed=0, n3=300, n4=100)
    R = raster.Rasterizer(scene.n3, scene.n4, views, capacity=1024)
    big = abi.splat_bins(1 << 28, R.keys.data_ptr(), R.vals.data_ptr(), R.ranges.data_ptr(),
                         R.n_instances.data_ptr())
    rc = abi.splat_bin_sort_noalloc(C.byref(R.cproj), R.cviews, R.V, C.byref(big), C.c_void_p(R.status.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == abi.SPLAT_ERR_CAPACITY
