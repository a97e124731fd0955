"""ctypes binding of libsplat (include/splat.h): struct mirrors and the entry
points under the same names.  Argument marshalling only -- every step of the
rasterizer runs in the CUDA library.  Importing this module fails loudly when
the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsplat.so")

SPLAT_OK = 0
SPLAT_ERR_INVALID_ARG = 1
SPLAT_ERR_CAPACITY = 2
SPLAT_ERR_TIMEOUT = 3
SPLAT_ERR_NONFINITE = 4
SPLAT_ERR_CUDA = 5

SPLAT_F32, SPLAT_BF16, SPLAT_F16 = 0, 1, 2
SPLAT_OP_BIN_SORT, SPLAT_OP_COMPOSITE_BWD, SPLAT_OP_CONVERT, SPLAT_OP_ALL, SPLAT_OP_CONVERT_STATE = 1, 2, 3, 4, 5
SPLAT_BWD_STOP_2D = 1
SPLAT_BWD_ADJOINT_ONLY = 2
SPLAT_MAX_VIEWS = 16
SPLAT_MAX_INSTANCES = 1 << 30
SPLAT_MAX_SH_TIME = 4
SPLAT_NOALLOC_SCRATCH_BYTES = 32 << 20

STAGES = {1: "slice_project", 2: "depth_sort", 3: "scan", 4: "duplicate", 5: "tile_sort",
          6: "composite_fwd", 7: "composite_bwd", 8: "adjoint", 9: "convert", 10: "densify"}


class splat_g3(C.Structure):
    _fields_ = [("n", C.c_int64), ("capacity", C.c_int64), ("dtype", C.c_int32), ("reserved", C.c_int32),
                ("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p)]


class splat_g4(C.Structure):
    _fields_ = [("n", C.c_int64), ("dtype", C.c_int32), ("sh_time", C.c_int32),
                ("mean", C.c_void_p), ("log_scale", C.c_void_p), ("ql", C.c_void_p), ("qr", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class splat_view(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("T", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("W", C.c_int32), ("H", C.c_int32), ("t", C.c_float),
                ("z_near", C.c_float), ("bg", C.c_float * 3), ("reserved", C.c_float)]


class splat_proj(C.Structure):
    _fields_ = [("n", C.c_int64), ("views", C.c_int32), ("reserved", C.c_int32),
                ("xy", C.c_void_p), ("conic_opacity", C.c_void_p), ("rgb_depth", C.c_void_p),
                ("rect", C.c_void_p), ("radius", C.c_void_p), ("n_tiles", C.c_void_p)]


class splat_bins(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("keys", C.c_void_p), ("vals", C.c_void_p), ("ranges", C.c_void_p),
                ("n_instances", C.c_void_p), ("tile_order", C.c_void_p), ("n_needed", C.c_void_p)]


class splat_image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("final_T", C.c_void_p), ("last", C.c_void_p)]


class splat_grads3(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p)]


class splat_grads4(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("ql", C.c_void_p), ("qr", C.c_void_p),
                ("opacity", C.c_void_p), ("sh", C.c_void_p)]


class splat_adam_set(C.Structure):
    _fields_ = [("param", C.c_void_p * 6), ("m", C.c_void_p * 6), ("v", C.c_void_p * 6)]


class splat_adam_hyper(C.Structure):
    _fields_ = [("lr3", C.c_float * 5), ("lr4", C.c_float * 6), ("lr_sh_rest", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("step", C.c_int32)]


class splat_options(C.Structure):
    _fields_ = [("pixels_per_lane_fwd", C.c_int32), ("pixels_per_lane_bwd", C.c_int32), ("tile_sort", C.c_int32),
                ("tile_cull", C.c_int32), ("spin_limit", C.c_int64), ("stats", C.c_void_p)]


def options(ppl_fwd=0, ppl_bwd=0, tile_sort=-1, tile_cull=-1, spin_limit=-1, stats=None) -> splat_options:
    """A splat_options whose unset fields take the library-wide defaults."""
    return splat_options(int(ppl_fwd), int(ppl_bwd), int(tile_sort), int(tile_cull), int(spin_limit), stats)


class splat_densify_rule(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("dense_scale", C.c_float), ("min_opacity", C.c_float),
                ("split_shrink", C.c_float)]


class splat_densify_set(C.Structure):
    _fields_ = [("n", C.c_int64), ("capacity", C.c_int64), ("state", C.POINTER(splat_adam_set)),
                ("accum", C.c_void_p), ("count", C.c_void_p), ("noise", C.c_void_p), ("sh_time", C.c_int32),
                ("reserved", C.c_int32)]


_P = C.POINTER
EXPORTS = {
    "splat_version": (C.c_int32, []),
    "splat_launch_count": (C.c_int64, []),
    "splat_set_spin_limit": (None, [C.c_int64]),
    "splat_set_pixels_per_lane": (None, [C.c_int, C.c_int]),
    "splat_set_tile_sort": (None, [C.c_int]),
    "splat_set_tile_cull": (None, [C.c_int]),
    "splat_set_stats": (None, [C.c_void_p]),
    "splat_status_string": (C.c_char_p, [C.c_int32]),
    "splat_total_tiles": (C.c_int64, [C.c_int, _P(C.c_int32), _P(C.c_int32)]),
    "splat_workspace_size": (C.c_size_t, [C.c_int, C.c_int64, C.c_int64, C.c_int, _P(C.c_int32), _P(C.c_int32),
                                          C.c_int64]),
    "splat_slice_project": (C.c_int, [_P(splat_g3), _P(splat_g4), _P(splat_view), C.c_int, _P(splat_proj),
                                      C.c_void_p, C.c_void_p]),
    "splat_bin_sort": (C.c_int, [_P(splat_proj), _P(splat_view), C.c_int, _P(splat_bins), C.c_void_p, C.c_void_p,
                                 C.c_size_t, C.c_void_p]),
    "splat_composite_fwd": (C.c_int, [_P(splat_proj), _P(splat_bins), _P(splat_view), C.c_int, _P(splat_image),
                                      C.c_void_p, C.c_void_p]),
    "splat_composite_fwd_l1": (C.c_int, [_P(splat_proj), _P(splat_bins), _P(splat_view), C.c_int, _P(splat_image),
                                         C.c_void_p, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "splat_composite_bwd": (C.c_int, [_P(splat_proj), _P(splat_bins), _P(splat_view), C.c_int, _P(splat_image),
                                      C.c_void_p, _P(splat_g3), _P(splat_g4), _P(splat_grads3), _P(splat_grads4),
                                      C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "splat_convert_4d_to_3d": (C.c_int, [_P(splat_g4), _P(splat_g3), C.c_float, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_size_t, C.c_void_p]),
    "splat_l1_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "splat_bin_sort_noalloc": (C.c_int, [_P(splat_proj), _P(splat_view), C.c_int, _P(splat_bins), C.c_void_p,
                                         C.c_void_p]),
    "splat_adam_step": (C.c_int, [_P(splat_adam_hyper), _P(splat_adam_set), _P(splat_grads3), _P(splat_g3),
                                  _P(splat_adam_set), _P(splat_grads4), _P(splat_g4), C.c_void_p, C.c_void_p]),
    "splat_cast_params": (C.c_int, [_P(splat_g3), _P(splat_g3), _P(splat_g4), _P(splat_g4), C.c_void_p]),
    "splat_convert_adam_state": (C.c_int, [_P(splat_g4), _P(splat_g3), C.c_float, _P(splat_adam_set),
                                           _P(splat_adam_set), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "splat_densify_stats": (C.c_int, [_P(splat_proj), _P(splat_view), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "splat_densify": (C.c_int, [_P(splat_densify_rule), _P(splat_densify_set), _P(splat_densify_set), C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "splat_densify_workspace_size": (C.c_size_t, [C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int]),
    "splat_workspace_size_4d": (C.c_size_t, [C.c_int, C.c_int64, C.c_int]),
    "splat_peak_probe": (C.c_double, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "splat_workspace_size_opts": (C.c_size_t, [C.c_int, C.c_int64, C.c_int64, C.c_int, _P(C.c_int32), _P(C.c_int32),
                                               C.c_int64, _P(splat_options)]),
    "splat_bin_sort_opts": (C.c_int, [_P(splat_proj), _P(splat_view), C.c_int, _P(splat_bins), C.c_void_p, C.c_void_p,
                                      C.c_size_t, _P(splat_options), C.c_void_p]),
    "splat_composite_fwd_opts": (C.c_int, [_P(splat_proj), _P(splat_bins), _P(splat_view), C.c_int, _P(splat_image),
                                           C.c_void_p, _P(splat_options), C.c_void_p]),
    "splat_composite_fwd_l1_opts": (C.c_int, [_P(splat_proj), _P(splat_bins), _P(splat_view), C.c_int,
                                              _P(splat_image), C.c_void_p, C.c_float, C.c_void_p, C.c_void_p,
                                              C.c_void_p, _P(splat_options), C.c_void_p]),
    "splat_composite_bwd_opts": (C.c_int, [_P(splat_proj), _P(splat_bins), _P(splat_view), C.c_int, _P(splat_image),
                                           C.c_void_p, _P(splat_g3), _P(splat_g4), _P(splat_grads3),
                                           _P(splat_grads4), C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                                           C.c_size_t, _P(splat_options), C.c_void_p]),
}

_lib = None


def lib():
    """The loaded libsplat (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsplat is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SplatError(RuntimeError):
    def __init__(self, code, where="", stage=0, aux=0):
        self.code, self.stage, self.aux = int(code), int(stage), int(aux)
        msg = "%s: %s" % (where, status_string(code))
        if stage:
            msg += " (stage %s, aux %d)" % (STAGES.get(stage, stage), aux)
        super().__init__(msg)


def status_string(code) -> str:
    return lib().splat_status_string(int(code)).decode()


def splat_status_string(code) -> str:
    return status_string(code)


def check(code, where):
    if code != SPLAT_OK:
        raise SplatError(code, where)


# --- entry points, same names as the C ABI ---------------------------------

def splat_version():
    return lib().splat_version()


def splat_launch_count():
    return lib().splat_launch_count()


def splat_set_spin_limit(n):
    lib().splat_set_spin_limit(int(n))


def splat_set_tile_sort(mode):
    lib().splat_set_tile_sort(int(mode))


def splat_set_stats(dev_counters_ptr):
    lib().splat_set_stats(dev_counters_ptr)


def splat_set_tile_cull(on):
    lib().splat_set_tile_cull(int(bool(on)))


def splat_set_pixels_per_lane(fwd, bwd):
    lib().splat_set_pixels_per_lane(int(fwd), int(bwd))


def _i32arr(vals):
    a = (C.c_int32 * max(1, len(vals)))(*[int(x) for x in vals])
    return a


def splat_total_tiles(W, H):
    return lib().splat_total_tiles(len(W), _i32arr(W), _i32arr(H))


def splat_workspace_size(op, N3, N4, W, H, capacity):
    return lib().splat_workspace_size(int(op), int(N3), int(N4), len(W), _i32arr(W), _i32arr(H), int(capacity))


def splat_slice_project(g3, g4, views, V, proj, status, stream):
    return lib().splat_slice_project(g3, g4, views, V, proj, status, stream)


def splat_bin_sort(proj, views, V, bins, status, ws, ws_bytes, stream):
    return lib().splat_bin_sort(proj, views, V, bins, status, ws, ws_bytes, stream)


def splat_composite_fwd(proj, bins, views, V, img, status, stream):
    return lib().splat_composite_fwd(proj, bins, views, V, img, status, stream)


def splat_composite_fwd_l1(proj, bins, views, V, img, target, scale, dL, loss, status, stream):
    return lib().splat_composite_fwd_l1(proj, bins, views, V, img, target, scale, dL, loss, status, stream)


def splat_composite_bwd(proj, bins, views, V, img, dL, g3, g4, dg3, dg4, dproj, flags, status, ws, ws_bytes, stream):
    return lib().splat_composite_bwd(proj, bins, views, V, img, dL, g3, g4, dg3, dg4, dproj, flags, status, ws,
                                     ws_bytes, stream)


def splat_convert_4d_to_3d(g4, g3, tau, n_moved, status, ws, ws_bytes, stream):
    return lib().splat_convert_4d_to_3d(g4, g3, tau, n_moved, status, ws, ws_bytes, stream)


def splat_l1_loss(img, target, n, scale, dL, loss, stream):
    return lib().splat_l1_loss(img, target, n, scale, dL, loss, stream)


def splat_bin_sort_noalloc(proj, views, V, bins, status, stream):
    """splat_bin_sort without a workspace argument, for callers that cannot
    allocate device memory when they sort (scratch: a fixed array inside the
    library, shared by all calls)."""
    return lib().splat_bin_sort_noalloc(proj, views, V, bins, status, stream)


def splat_adam_step(hyper, s3, dg3, g3, s4, dg4, g4, status, stream):
    return lib().splat_adam_step(hyper, s3, dg3, g3, s4, dg4, g4, status, stream)


def splat_cast_params(src3, dst3, src4, dst4, stream):
    return lib().splat_cast_params(src3, dst3, src4, dst4, stream)


def splat_convert_adam_state(g4, g3, tau, s4, s3, status, ws, ws_bytes, stream):
    return lib().splat_convert_adam_state(g4, g3, tau, s4, s3, status, ws, ws_bytes, stream)


def splat_densify_stats(proj, views, V, dproj, accum, count, stream):
    return lib().splat_densify_stats(proj, views, V, dproj, accum, count, stream)


def splat_densify(rule, set3, set4, n_out, status, ws, ws_bytes, stream):
    return lib().splat_densify(rule, set3, set4, n_out, status, ws, ws_bytes, stream)


def splat_densify_workspace_size(n3, cap3, n4, cap4, sh_time4=0):
    return int(lib().splat_densify_workspace_size(int(n3), int(cap3), int(n4), int(cap4), int(sh_time4)))


def splat_workspace_size_4d(op, N4, sh_time):
    return int(lib().splat_workspace_size_4d(int(op), int(N4), int(sh_time)))


SPLAT_PROBE_FFMA, SPLAT_PROBE_FFMA2, SPLAT_PROBE_EX2, SPLAT_PROBE_RCP = 0, 1, 2, 3


def splat_peak_probe(kind, blocks, iters, out, stream):
    """Launches one pipe-throughput probe; returns its operation count (-1 on error)."""
    return float(lib().splat_peak_probe(int(kind), int(blocks), int(iters), out, stream))


def splat_workspace_size_opts(op, N3, N4, W, H, capacity, opt):
    return lib().splat_workspace_size_opts(int(op), int(N3), int(N4), len(W), _i32arr(W), _i32arr(H), int(capacity),
                                           opt)


def splat_bin_sort_opts(proj, views, V, bins, status, ws, ws_bytes, opt, stream):
    return lib().splat_bin_sort_opts(proj, views, V, bins, status, ws, ws_bytes, opt, stream)


def splat_composite_fwd_opts(proj, bins, views, V, img, status, opt, stream):
    return lib().splat_composite_fwd_opts(proj, bins, views, V, img, status, opt, stream)


def splat_composite_fwd_l1_opts(proj, bins, views, V, img, target, scale, dL, loss, status, opt, stream):
    return lib().splat_composite_fwd_l1_opts(proj, bins, views, V, img, target, scale, dL, loss, status, opt, stream)


def splat_composite_bwd_opts(proj, bins, views, V, img, dL, g3, g4, dg3, dg4, dproj, flags, status, ws, ws_bytes, opt,
                             stream):
    return lib().splat_composite_bwd_opts(proj, bins, views, V, img, dL, g3, g4, dg3, dg4, dproj, flags, status, ws,
                                          ws_bytes, opt, stream)
