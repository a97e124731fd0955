"""PyTorch front end of libsplat: device buffers, streams, autograd and CUDA graphs.

PyTorch supplies device memory and streams only; every stage of the
rasterizer (slice/project, bin/sort, composite forward/backward, adjoint,
4D->3D conversion, L1 loss) is a libsplat kernel reached through the C ABI.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import abi
from .abi import SplatError

FIELDS3 = ("mean3", "log_scale3", "quat3", "opacity3", "sh3")
FIELDS4 = ("mean4", "log_scale4", "ql", "qr", "opacity4", "sh4")
SHAPES = {"mean3": (3,), "log_scale3": (3,), "quat3": (4,), "opacity3": (), "sh3": (16, 3),
          "mean4": (4,), "log_scale4": (4,), "ql": (4,), "qr": (4,), "opacity4": (), "sh4": (16, 3)}


def shape_of(k: str, sh_time: int = 0):
    """Per-row shape of field k; a 4D colour with sh_time time frequencies holds
    a block of 16 x 3 coefficients per frequency."""
    return (16 * (sh_time + 1), 3) if k == "sh4" else SHAPES[k]

_DTYPES = {torch.float32: abi.SPLAT_F32, torch.bfloat16: abi.SPLAT_BF16, torch.float16: abi.SPLAT_F16}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Gaussians:
    """One hybrid parameter set on the device: static 3D and dynamic 4D Gaussians,
    raw (pre-activation) values in a storage dtype (float32, bfloat16 or float16).
    The 3D arrays have `capacity3` rows so that 4D->3D conversion can append."""

    def __init__(self, t: Dict[str, torch.Tensor], n3: int, n4: int):
        self.t = t
        self.n3, self.n4 = int(n3), int(n4)
        dt = t["mean3"].dtype
        if any(t[k].dtype != dt for k in FIELDS3 + FIELDS4):
            raise ValueError("all fields must share one dtype")
        self.dtype = dt
        self.code = _DTYPES[dt]
        self.sh_time = int(t["sh4"].shape[1]) // 16 - 1 if t["sh4"].dim() == 3 else 0

    @property
    def capacity3(self) -> int:
        return int(self.t["mean3"].shape[0])

    @property
    def capacity4(self) -> int:
        return int(self.t["mean4"].shape[0])

    @property
    def n(self) -> int:
        return self.n3 + self.n4

    @classmethod
    def from_scene(cls, scene, device="cuda", dtype=torch.float32, capacity3: Optional[int] = None,
                   capacity4: Optional[int] = None) -> "Gaussians":
        cap = scene.n3 if capacity3 is None else max(int(capacity3), scene.n3)
        cap4 = scene.n4 if capacity4 is None else max(int(capacity4), scene.n4)
        t = {}
        for k in FIELDS3 + FIELDS4:
            a = torch.from_numpy(np.ascontiguousarray(getattr(scene, k), dtype=np.float32))
            rows, n = (cap, scene.n3) if k in FIELDS3 else (cap4, scene.n4)
            if rows > n:
                pad = torch.zeros((rows - n,) + tuple(a.shape[1:]), dtype=torch.float32)
                a = torch.cat([a, pad], 0)
            t[k] = a.to(device=device, dtype=dtype).contiguous()
        return cls(t, scene.n3, scene.n4)

    def dequantised(self) -> Dict[str, np.ndarray]:
        """The stored values as float64 host arrays (first n rows)."""
        out = {}
        for k in FIELDS3:
            out[k] = self.t[k][: self.n3].float().cpu().double().numpy()
        for k in FIELDS4:
            out[k] = self.t[k][: self.n4].float().cpu().double().numpy()
        return out

    def c_g3(self) -> abi.splat_g3:
        t = self.t
        return abi.splat_g3(self.n3, self.capacity3, self.code, 0, t["mean3"].data_ptr(), t["log_scale3"].data_ptr(),
                            t["quat3"].data_ptr(), t["opacity3"].data_ptr(), t["sh3"].data_ptr())

    def c_g4(self) -> abi.splat_g4:
        t = self.t
        return abi.splat_g4(self.n4, self.code, self.sh_time, t["mean4"].data_ptr(), t["log_scale4"].data_ptr(),
                            t["ql"].data_ptr(), t["qr"].data_ptr(), t["opacity4"].data_ptr(), t["sh4"].data_ptr())


def c_views(views) -> "C.Array":
    arr = (abi.splat_view * len(views))()
    for i, v in enumerate(views):
        R = np.asarray(v.R, dtype=np.float32).reshape(9)
        T = np.asarray(v.T, dtype=np.float32).reshape(3)
        s = arr[i]
        for k in range(9):
            s.R[k] = float(R[k])
        for k in range(3):
            s.T[k] = float(T[k])
            s.bg[k] = float(v.bg[k])
        s.fx, s.fy, s.cx, s.cy = float(v.fx), float(v.fy), float(v.cx), float(v.cy)
        s.W, s.H = int(v.W), int(v.H)
        s.t = float(v.t)
        s.z_near = float(v.z_near)
    return arr


class Rasterizer:
    """Owns the device buffers of one (Gaussian count, view batch) shape and runs
    the pipeline on a CUDA stream.  All V views are rendered by one launch per
    stage.  `capacity` is the tile-instance capacity; `None` picks it from a
    first render (see `autotune_capacity`)."""

    def __init__(self, n3: int, n4: int, views: Sequence, device="cuda", capacity: Optional[int] = None,
                 headroom: float = 1.25, keep_keys: bool = True, sh_time: int = 0):
        self.keep_keys = keep_keys
        # this rasterizer's tuning (splat_options): unset fields follow the
        # library-wide splat_set_* defaults; see set_options
        self.options = abi.options()
        self.n3, self.n4 = int(n3), int(n4)
        self.N = self.n3 + self.n4
        self.views = list(views)
        self.V = len(self.views)
        if not 1 <= self.V <= abi.SPLAT_MAX_VIEWS:
            raise ValueError("1..%d views per batch" % abi.SPLAT_MAX_VIEWS)
        self.device = torch.device(device)
        self.cviews = c_views(self.views)
        self.W = [int(v.W) for v in self.views]
        self.H = [int(v.H) for v in self.views]
        self.total_tiles = abi.splat_total_tiles(self.W, self.H)
        self.pix = [w * h for w, h in zip(self.W, self.H)]
        self.pix_base = np.concatenate([[0], np.cumsum(self.pix)]).astype(np.int64)
        self.headroom = headroom
        rows = self.V * self.N
        d, f32, i32 = self.device, torch.float32, torch.int32
        self.xy = torch.zeros((rows, 2), dtype=f32, device=d)
        self.conic_opacity = torch.zeros((rows, 4), dtype=f32, device=d)
        self.rgb_depth = torch.zeros((rows, 4), dtype=f32, device=d)
        self.rect = torch.zeros((rows, 4), dtype=i32, device=d)
        self.radius = torch.zeros((rows,), dtype=i32, device=d)
        self.n_tiles = torch.zeros((rows,), dtype=i32, device=d)
        self.cproj = abi.splat_proj(self.N, self.V, 0, self.xy.data_ptr(), self.conic_opacity.data_ptr(),
                                    self.rgb_depth.data_ptr(), self.rect.data_ptr(), self.radius.data_ptr(),
                                    self.n_tiles.data_ptr())
        total_pix = int(self.pix_base[-1])
        self.rgb = torch.zeros((3 * total_pix,), dtype=f32, device=d)
        self.final_T = torch.zeros((total_pix,), dtype=f32, device=d)
        self.last = torch.zeros((total_pix,), dtype=i32, device=d)
        self.cimg = abi.splat_image(self.rgb.data_ptr(), self.final_T.data_ptr(), self.last.data_ptr())
        self.status = torch.zeros((4,), dtype=i32, device=d)
        self.n_instances = torch.zeros((1,), dtype=torch.int64, device=d)
        self.n_needed = torch.zeros((1,), dtype=torch.int64, device=d)  # capacity the last sort needed
        self.ranges = torch.zeros((max(1, self.total_tiles) * 2,), dtype=i32, device=d)
        # tiles longest list first, for the compositing kernels' scheduling
        self.tile_order = torch.arange(max(1, self.total_tiles), dtype=i32, device=d)
        self.dproj = torch.zeros((rows * 12,), dtype=f32, device=d)
        self.loss = torch.zeros((1,), dtype=f32, device=d)
        self.dL = torch.zeros_like(self.rgb)
        # gradient rows for N Gaussians in either set, so that the 3D / 4D split can
        # change (4D -> 3D conversion) without reallocating; self.grads views the first n
        self.sh_time = int(sh_time)
        self._grad_buf = {k: torch.zeros((self.N,) + shape_of(k, self.sh_time), dtype=f32, device=d)
                          for k in FIELDS3 + FIELDS4}
        self.cg3 = abi.splat_grads3(*[self._grad_buf[k].data_ptr() for k in FIELDS3])
        self.cg4 = abi.splat_grads4(*[self._grad_buf[k].data_ptr() for k in FIELDS4])
        self._view_grads()
        if capacity is None:
            capacity = max(1 << 16, 16 * rows)
        self.set_capacity(capacity)

    # -- buffers ------------------------------------------------------------
    def _view_grads(self):
        self.grads = {k: self._grad_buf[k][: (self.n3 if k in FIELDS3 else self.n4)] for k in FIELDS3 + FIELDS4}

    def set_counts(self, n3: int, n4: int):
        """New 3D / 4D split of the same N Gaussians (after a 4D -> 3D conversion)."""
        if int(n3) + int(n4) != self.N:
            raise ValueError("the split must keep N = %d" % self.N)
        self.n3, self.n4 = int(n3), int(n4)
        self._view_grads()

    def set_views(self, views: Sequence):
        """New cameras / timestamps for the next calls; resolutions must stay the same."""
        views = list(views)
        if len(views) != self.V or any((int(v.W), int(v.H)) != (w, h) for v, w, h in zip(views, self.W, self.H)):
            raise ValueError("set_views keeps the batch's count and resolutions")
        self.views = views
        self.cviews = c_views(views)

    def set_capacity(self, capacity: int):
        capacity = int(min(max(1, capacity), abi.SPLAT_MAX_INSTANCES))
        self.capacity = capacity
        self.keys = torch.empty((capacity if self.keep_keys else 0,), dtype=torch.int32, device=self.device)
        self.vals = torch.empty((capacity,), dtype=torch.int32, device=self.device)
        self.cbins = abi.splat_bins(capacity, self.keys.data_ptr() if self.keep_keys else None, self.vals.data_ptr(),
                                    self.ranges.data_ptr(), self.n_instances.data_ptr(), self.tile_order.data_ptr(),
                                    self.n_needed.data_ptr())
        ws = abi.splat_workspace_size_opts(abi.SPLAT_OP_ALL, self.n3, self.n4, self.W, self.H, capacity,
                                           C.byref(self.options))
        if ws == 0:
            raise ValueError("invalid sizes for the workspace")
        self.ws_bytes = int(ws)
        self.ws = torch.empty((self.ws_bytes,), dtype=torch.uint8, device=self.device)

    def set_options(self, ppl_fwd=None, ppl_bwd=None, tile_sort=None, tile_cull=None, spin_limit=None,
                    stats=False):
        """This rasterizer's tuning, independent of other rasterizers in the
        process: pixels per lane of the compositing kernels (2, 4, 8; 0 = the
        library default), tile sort mode and footprint culling of the sort (-1 =
        the library default), the bounded waits' spin limit (-1 = default) and
        the pair-count statistics (a device pointer, or None for the default).
        Arguments left out keep their current value."""
        o = self.options
        if ppl_fwd is not None:
            o.pixels_per_lane_fwd = int(ppl_fwd)
        if ppl_bwd is not None:
            o.pixels_per_lane_bwd = int(ppl_bwd)
        if spin_limit is not None:
            o.spin_limit = int(spin_limit)
        if stats is not False:
            o.stats = stats
        if tile_cull is not None:
            o.tile_cull = int(tile_cull)
        if tile_sort is not None and int(tile_sort) != o.tile_sort:
            o.tile_sort = int(tile_sort)
            self.set_capacity(self.capacity)  # the sort's workspace depends on the mode

    # -- stages -------------------------------------------------------------
    def slice_project(self, G: Gaussians, stream=None):
        if G.n3 != self.n3 or G.n4 != self.n4:
            raise ValueError("Gaussian counts differ from the rasterizer's")
        if G.sh_time != self.sh_time:
            raise ValueError("the 4D colour's time frequencies differ from the rasterizer's")
        g3, g4 = G.c_g3(), G.c_g4()
        abi.check(abi.splat_slice_project(C.byref(g3), C.byref(g4), self.cviews, self.V, C.byref(self.cproj),
                                          _ptr(self.status), _stream(stream)), "splat_slice_project")

    def bin_sort(self, stream=None):
        abi.check(abi.splat_bin_sort_opts(C.byref(self.cproj), self.cviews, self.V, C.byref(self.cbins),
                                          _ptr(self.status), _ptr(self.ws), self.ws_bytes, C.byref(self.options),
                                          _stream(stream)), "splat_bin_sort")

    def composite(self, stream=None):
        abi.check(abi.splat_composite_fwd_opts(C.byref(self.cproj), C.byref(self.cbins), self.cviews, self.V,
                                               C.byref(self.cimg), _ptr(self.status), C.byref(self.options),
                                               _stream(stream)), "splat_composite_fwd")

    def forward(self, G: Gaussians, stream=None):
        """Slice/project, bin/sort and composite all views (asynchronous)."""
        self.slice_project(G, stream)
        self.bin_sort(stream)
        self.composite(stream)
        return self.rgb

    def _bwd(self, G: Gaussians, dL_drgb: Optional[torch.Tensor], flags: int, stream=None):
        g3, g4 = G.c_g3(), G.c_g4()
        abi.check(abi.splat_composite_bwd_opts(C.byref(self.cproj), C.byref(self.cbins), self.cviews, self.V,
                                               C.byref(self.cimg), _ptr(dL_drgb), C.byref(g3), C.byref(g4),
                                               C.byref(self.cg3), C.byref(self.cg4), _ptr(self.dproj), flags,
                                               _ptr(self.status), _ptr(self.ws), self.ws_bytes, C.byref(self.options),
                                               _stream(stream)), "splat_composite_bwd")

    def backward(self, G: Gaussians, dL_drgb: torch.Tensor, stream=None, stop_2d: bool = False):
        """Gradients of all parameters for pixel gradient dL_drgb (asynchronous);
        results in self.grads (overwritten) and self.dproj."""
        self._bwd(G, dL_drgb, abi.SPLAT_BWD_STOP_2D if stop_2d else 0, stream)
        return self.grads

    def adjoint(self, G: Gaussians, stream=None):
        """Chain self.dproj through the projection into self.grads (asynchronous)."""
        self._bwd(G, None, abi.SPLAT_BWD_ADJOINT_ONLY, stream)
        return self.grads

    def l1_loss(self, target: torch.Tensor, stream=None):
        """L1 loss (mean over pixels and channels) and its pixel gradient into self.dL."""
        n = self.rgb.numel()
        abi.check(abi.splat_l1_loss(_ptr(self.rgb), _ptr(target), n, 1.0 / max(1, n), _ptr(self.dL),
                                    _ptr(self.loss), _stream(stream)), "splat_l1_loss")
        return self.loss

    def composite_l1(self, target: torch.Tensor, stream=None):
        """Composite all views with the L1 loss fused in (the same image, loss and
        pixel gradient as composite() followed by l1_loss(); asynchronous)."""
        n = self.rgb.numel()
        abi.check(abi.splat_composite_fwd_l1_opts(C.byref(self.cproj), C.byref(self.cbins), self.cviews, self.V,
                                                  C.byref(self.cimg), _ptr(target), 1.0 / max(1, n), _ptr(self.dL),
                                                  _ptr(self.loss), _ptr(self.status), C.byref(self.options),
                                                  _stream(stream)), "splat_composite_fwd_l1")
        return self.loss

    STAGES = ("slice_project", "bin_sort", "composite_fwd", "loss", "composite_bwd", "adjoint")
    fuse_loss = True  # step(): the L1 loss inside the forward compositing (the "loss" stage is then empty)

    def step(self, G: Gaussians, target: torch.Tensor, stream=None, marks: Optional[dict] = None):
        """One training step of the rasterizer over the whole view batch: forward,
        L1 loss, backward.  `marks` (optional) maps "start" and each name of
        STAGES to a CUDA event recorded after that stage."""
        st = torch.cuda.current_stream() if stream is None else stream

        def mark(name):
            if marks is not None:
                marks[name].record(st)

        mark("start")
        self.slice_project(G, stream)
        mark("slice_project")
        self.bin_sort(stream)
        mark("bin_sort")
        if self.fuse_loss:
            self.composite_l1(target, stream)
            mark("composite_fwd")
        else:
            self.composite(stream)
            mark("composite_fwd")
            self.l1_loss(target, stream)
        mark("loss")
        self._bwd(G, self.dL, abi.SPLAT_BWD_STOP_2D, stream)
        mark("composite_bwd")
        self._bwd(G, None, abi.SPLAT_BWD_ADJOINT_ONLY, stream)
        mark("adjoint")

    # -- status / capacity -------------------------------------------------
    def read_status(self):
        """Synchronising read of the device status word."""
        s = self.status.cpu().numpy()
        aux = (int(s[3]) << 32) | (int(s[2]) & 0xFFFFFFFF)
        return int(s[0]), int(s[1]), aux

    def check(self, where="rasterizer"):
        code, stage, aux = self.read_status()
        if code != abi.SPLAT_OK:
            raise SplatError(code, where, stage, aux)

    def instances(self) -> int:
        return int(self.n_instances.item())

    def autotune_capacity(self, G: Gaussians, retries: int = 5) -> int:
        """Render once; when the instance list overflows, grow it to the required
        count times the headroom and render again.  Returns K."""
        for _ in range(retries):
            self.forward(G)
            code, stage, aux = self.read_status()
            if code == abi.SPLAT_ERR_CAPACITY:
                self.set_capacity(int(math.ceil(aux * self.headroom)) + 1024)
                continue
            if code != abi.SPLAT_OK:
                raise SplatError(code, "autotune_capacity", stage, aux)
            K = self.instances()
            # the super-tile lists of the binned sort share the capacity
            want = int(math.ceil(max(K, int(self.n_needed.item())) * self.headroom)) + 1024
            if want < self.capacity // 2 or want > self.capacity:
                self.set_capacity(want)
            return K
        raise SplatError(abi.SPLAT_ERR_CAPACITY, "autotune_capacity")

    # -- views of the flat buffers -----------------------------------------
    def image(self, v: int, buf: Optional[torch.Tensor] = None) -> torch.Tensor:
        b = self.rgb if buf is None else buf
        p0 = int(self.pix_base[v])
        return b[3 * p0: 3 * p0 + 3 * self.pix[v]].view(3, self.H[v], self.W[v])

    def plane(self, v: int, buf: torch.Tensor) -> torch.Tensor:
        p0 = int(self.pix_base[v])
        return buf[p0: p0 + self.pix[v]].view(self.H[v], self.W[v])


def stage_events(external: bool = False) -> dict:
    kw = {"enable_timing": True}
    if external:
        kw["external"] = True
    return {k: torch.cuda.Event(**kw) for k in ("start",) + Rasterizer.STAGES}


class GraphedStep:
    """CUDA graphs of one full rasterizer training step (forward, L1 loss,
    backward) over the whole view batch: one replay launches every kernel of
    the step with no host work in between.  With copies > 1 several identical
    graphs are captured, each recording its own per-stage events, so that a
    run of consecutive replays can be broken down by stage afterwards."""

    def __init__(self, R: Rasterizer, G: Gaussians, target: torch.Tensor, warmup: int = 2, copies: int = 1,
                 with_marks: bool = False):
        self.R, self.G, self.target = R, G, target
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                R.step(G, target, s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        R.check("GraphedStep warm-up")
        self.graphs, self.marks = [], []
        n0 = abi.lib().splat_launch_count()
        for _ in range(max(1, copies)):
            g = torch.cuda.CUDAGraph()
            marks = stage_events(external=True) if with_marks else None
            with torch.cuda.graph(g):
                R.step(G, target, marks=marks)
            self.graphs.append(g)
            self.marks.append(marks)
        self.launches_per_step = (abi.lib().splat_launch_count() - n0) // max(1, copies)
        self.graph = self.graphs[0]

    def replay(self, i: int = 0):
        self.graphs[i % len(self.graphs)].replay()

    def stage_ms(self, i: int) -> dict:
        m = self.marks[i]
        names = ("start",) + Rasterizer.STAGES
        return {b: m[a].elapsed_time(m[b]) for a, b in zip(names[:-1], names[1:])}


class HybridRasterize(torch.autograd.Function):
    """autograd entry: HybridRasterize.apply(R, G, *param_tensors) -> flat rgb of
    all views.  The parameter tensors must be the ones held by G (11 of them,
    3D fields first); gradients come from the hand-written adjoint kernels."""

    @staticmethod
    def forward(ctx, R: Rasterizer, G: Gaussians, *params):
        R.forward(G)
        ctx.R, ctx.G = R, G
        return R.rgb.clone()

    @staticmethod
    def backward(ctx, grad_rgb):
        R, G = ctx.R, ctx.G
        R.backward(G, grad_rgb.contiguous())
        out = [None, None]
        for k in FIELDS3:
            g = torch.zeros_like(G.t[k], dtype=torch.float32)
            g[: G.n3] = R.grads[k]
            out.append(g.to(G.t[k].dtype))
        for k in FIELDS4:
            out.append(R.grads[k].clone().to(G.t[k].dtype))
        return tuple(out)


def render(G: Gaussians, views, capacity=None) -> List[torch.Tensor]:
    """Convenience: render the views, return [3, H, W] images (synchronises)."""
    R = Rasterizer(G.n3, G.n4, views, device=G.t["mean3"].device, capacity=capacity, sh_time=G.sh_time)
    R.autotune_capacity(G)
    R.forward(G)
    R.check("render")
    return [R.image(v).clone() for v in range(R.V)]


def convert_4d_to_3d(G: Gaussians, tau: float, stream=None) -> int:
    """Sec. 4.1-4.2 in place on G: moves every 4D Gaussian with exp(s_t) > tau to the
    3D set (appending within capacity3) and compacts the 4D set.  Synchronises
    once to read the moved count.  Returns the number moved."""
    dev = G.t["mean3"].device
    bytes_ = max(256, abi.splat_workspace_size_4d(abi.SPLAT_OP_CONVERT, G.n4, G.sh_time))
    ws = torch.empty((int(bytes_),), dtype=torch.uint8, device=dev)
    status = torch.zeros((4,), dtype=torch.int32, device=dev)
    n_moved = torch.zeros((1,), dtype=torch.int64, device=dev)
    g3, g4 = G.c_g3(), G.c_g4()
    abi.check(abi.splat_convert_4d_to_3d(C.byref(g4), C.byref(g3), float(tau), _ptr(n_moved), _ptr(status),
                                         _ptr(ws), int(bytes_), _stream(stream)), "splat_convert_4d_to_3d")
    s = status.cpu().numpy()
    if s[0] != 0:
        raise SplatError(int(s[0]), "splat_convert_4d_to_3d", int(s[1]), (int(s[3]) << 32) | (int(s[2]) & 0xFFFFFFFF))
    m = int(n_moved.item())
    G.n3 += m
    G.n4 -= m
    return m
