"""C-ABI library checks that need no GPU: it loads, exports every symbol that
include/splat.h declares (under the same names in the Python binding), and
its host-side logic (sizes, argument checks, status strings) behaves."""
import ctypes as C
import os
import re

import pytest

from paper_2505_13215_gb300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "splat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(splat_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_13215_gb300 import build
    build.build()
    return abi.lib()


def test_header_declares_the_pipeline():
    names = declared_functions()
    for n in ("splat_slice_project", "splat_bin_sort", "splat_composite_fwd", "splat_composite_bwd",
              "splat_convert_4d_to_3d", "splat_workspace_size", "splat_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in abi.EXPORTS, name
        assert callable(getattr(abi, name, None)), "python binding lacks %s" % name


def test_status_strings(lib):
    for code in range(6):
        assert abi.status_string(code) != "unknown status"
    assert abi.status_string(99) == "unknown status"


def test_total_tiles_and_workspace(lib):
    assert abi.splat_total_tiles([1352], [1014]) == 85 * 64
    assert abi.splat_total_tiles([1352, 676], [1014, 507]) == 85 * 64 + 43 * 32
    a = abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, 200000, 100000, [1352], [1014], 30_000_000)
    b = abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, 200000, 100000, [1352], [1014], 60_000_000)
    assert 0 < a < b
    assert abi.splat_workspace_size(abi.SPLAT_OP_ALL, 10, 10, [64], [64], 1000) >= \
        abi.splat_workspace_size(abi.SPLAT_OP_COMPOSITE_BWD, 10, 10, [64], [64], 1000)
    # invalid: capacity above the limit, no views, unknown op
    assert abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, 1, 1, [64], [64], abi.SPLAT_MAX_INSTANCES + 1) == 0
    assert abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, 1, 1, [], [], 10) == 0
    assert abi.splat_workspace_size(17, 1, 1, [64], [64], 10) == 0


def test_invalid_arguments_rejected_before_any_device_work(lib):
    v = (abi.splat_view * 1)()
    v[0].W, v[0].H, v[0].fx, v[0].fy, v[0].z_near = 64, 64, 50.0, 50.0, 0.2
    proj = abi.splat_proj(0, 1, 0, None, None, None, None, None, None)
    g3 = abi.splat_g3()
    g4 = abi.splat_g4()
    st = C.c_void_p(0)
    # no status buffer
    assert abi.splat_slice_project(C.byref(g3), C.byref(g4), v, 1, C.byref(proj), st, None) == abi.SPLAT_ERR_INVALID_ARG
    # zero views / too many views
    assert abi.splat_slice_project(C.byref(g3), C.byref(g4), v, 0, C.byref(proj), C.c_void_p(16), None) == \
        abi.SPLAT_ERR_INVALID_ARG
    # image size out of range
    v[0].W = 0
    assert abi.splat_slice_project(C.byref(g3), C.byref(g4), v, 1, C.byref(proj), C.c_void_p(16), None) == \
        abi.SPLAT_ERR_INVALID_ARG
    v[0].W = 64
    # mixed storage dtypes
    g3.n, g3.capacity, g3.dtype = 1, 1, abi.SPLAT_F32
    g4.n, g4.dtype = 1, abi.SPLAT_BF16
    for f in ("mean", "log_scale", "quat", "opacity", "sh"):
        setattr(g3, f, 256)
    for f in ("mean", "log_scale", "ql", "qr", "opacity", "sh"):
        setattr(g4, f, 256)
    proj.n = 2
    assert abi.splat_slice_project(C.byref(g3), C.byref(g4), v, 1, C.byref(proj), C.c_void_p(16), None) == \
        abi.SPLAT_ERR_INVALID_ARG
    # convert: non-finite tau
    assert abi.splat_convert_4d_to_3d(C.byref(g4), C.byref(g3), float("nan"), C.c_void_p(16), C.c_void_p(16),
                                      None, 0, None) == abi.SPLAT_ERR_INVALID_ARG
    # loss: misaligned
    assert abi.splat_l1_loss(C.c_void_p(4), C.c_void_p(16), 8, 1.0, C.c_void_p(16), C.c_void_p(16), None) == \
        abi.SPLAT_ERR_INVALID_ARG


def test_knobs_are_host_side(lib):
    abi.splat_set_spin_limit(123)
    abi.splat_set_spin_limit(1 << 22)
    abi.splat_set_pixels_per_lane(3, 5)  # ignored
    abi.splat_set_pixels_per_lane(8, 8)
    assert abi.splat_version() == 0x000100


@pytest.mark.parametrize("missing", ["xy", "conic_opacity", "rgb_depth", "rect", "radius", "n_tiles"])
def test_both_bin_sorts_reject_the_same_projected_rows(lib, missing):
    """splat_bin_sort and splat_bin_sort_noalloc check their arguments alike:
    a projected-row array left NULL with rows present (the tile passes read xy
    and conic_opacity when footprint culling is on) is rejected on the host,
    before any device work; so are misaligned ranges / n_instances."""
    v = (abi.splat_view * 1)()
    v[0].W, v[0].H, v[0].fx, v[0].fy, v[0].z_near = 64, 64, 50.0, 50.0, 0.2
    fields = {f: 4096 for f in ("xy", "conic_opacity", "rgb_depth", "rect", "radius", "n_tiles")}
    fields[missing] = None
    proj = abi.splat_proj(10, 1, 0, fields["xy"], fields["conic_opacity"], fields["rgb_depth"], fields["rect"],
                          fields["radius"], fields["n_tiles"])
    bins = abi.splat_bins(1024, 4096, 4096, 4096, 4096)
    st = C.c_void_p(4096)
    assert abi.splat_bin_sort_noalloc(C.byref(proj), v, 1, C.byref(bins), st, None) == abi.SPLAT_ERR_INVALID_ARG
    assert abi.splat_bin_sort(C.byref(proj), v, 1, C.byref(bins), st, C.c_void_p(4096), 1 << 30, None) == \
        abi.SPLAT_ERR_INVALID_ARG


def test_both_bin_sorts_reject_misaligned_bins(lib):
    v = (abi.splat_view * 1)()
    v[0].W, v[0].H, v[0].fx, v[0].fy, v[0].z_near = 64, 64, 50.0, 50.0, 0.2
    proj = abi.splat_proj(10, 1, 0, 4096, 4096, 4096, 4096, 4096, 4096)
    st = C.c_void_p(4096)
    for ranges, n_inst in ((4100, 4096), (4096, 4100)):
        bins = abi.splat_bins(1024, 4096, 4096, ranges, n_inst)
        assert abi.splat_bin_sort_noalloc(C.byref(proj), v, 1, C.byref(bins), st, None) == abi.SPLAT_ERR_INVALID_ARG
        assert abi.splat_bin_sort(C.byref(proj), v, 1, C.byref(bins), st, C.c_void_p(4096), 1 << 30, None) == \
            abi.SPLAT_ERR_INVALID_ARG
    # a non-positive focal length is rejected by both, as by every entry point
    v[0].fx = 0.0
    bins = abi.splat_bins(1024, 4096, 4096, 4096, 4096)
    assert abi.splat_bin_sort_noalloc(C.byref(proj), v, 1, C.byref(bins), st, None) == abi.SPLAT_ERR_INVALID_ARG


def test_invalid_options_rejected_before_any_device_work(lib):
    """Per-call options (splat_options): out-of-range fields are rejected on the
    host; a NULL pointer or the library-default values are accepted."""
    W, H = [64], [64]
    base = abi.splat_workspace_size(abi.SPLAT_OP_BIN_SORT, 10, 10, W, H, 1000)
    assert abi.splat_workspace_size_opts(abi.SPLAT_OP_BIN_SORT, 10, 10, W, H, 1000, None) == base
    assert abi.splat_workspace_size_opts(abi.SPLAT_OP_BIN_SORT, 10, 10, W, H, 1000, C.byref(abi.options())) == base
    # the radix mode lays out its own workspace
    assert abi.splat_workspace_size_opts(abi.SPLAT_OP_BIN_SORT, 10, 10, W, H, 1000,
                                         C.byref(abi.options(tile_sort=1))) not in (0, base)
    for bad in (abi.options(ppl_fwd=3), abi.options(ppl_bwd=16), abi.options(tile_sort=3),
                abi.options(tile_cull=2), abi.options(spin_limit=-2)):
        assert abi.splat_workspace_size_opts(abi.SPLAT_OP_BIN_SORT, 10, 10, W, H, 1000, C.byref(bad)) == 0
    v = (abi.splat_view * 1)()
    v[0].W, v[0].H, v[0].fx, v[0].fy, v[0].z_near = 64, 64, 50.0, 50.0, 0.2
    proj = abi.splat_proj(10, 1, 0, 4096, 4096, 4096, 4096, 4096, 4096)
    bins = abi.splat_bins(1024, 4096, 4096, 4096, 4096)
    img = abi.splat_image(4096, 4096, 4096)
    st = C.c_void_p(4096)
    bad = abi.options(ppl_fwd=5)
    assert abi.splat_bin_sort_opts(C.byref(proj), v, 1, C.byref(bins), st, C.c_void_p(4096), 1 << 30,
                                   C.byref(abi.options(tile_sort=7)), None) == abi.SPLAT_ERR_INVALID_ARG
    assert abi.splat_composite_fwd_opts(C.byref(proj), C.byref(bins), v, 1, C.byref(img), st, C.byref(bad),
                                        None) == abi.SPLAT_ERR_INVALID_ARG
    assert abi.splat_composite_fwd_l1_opts(C.byref(proj), C.byref(bins), v, 1, C.byref(img), C.c_void_p(4096), 1.0,
                                           C.c_void_p(4096), C.c_void_p(4096), st, C.byref(bad),
                                           None) == abi.SPLAT_ERR_INVALID_ARG
    assert abi.splat_composite_bwd_opts(C.byref(proj), C.byref(bins), v, 1, C.byref(img), C.c_void_p(4096), None,
                                        None, None, None, None, abi.SPLAT_BWD_STOP_2D, st, C.c_void_p(4096), 1 << 30,
                                        C.byref(abi.options(ppl_bwd=1)), None) == abi.SPLAT_ERR_INVALID_ARG
