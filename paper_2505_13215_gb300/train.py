"""Training step of the hybrid 3D-4D representation on the GPU (Sec. 4.3).

One step renders a batch of views (cameras and timestamps) in one launch per
stage, takes the L1 loss against the targets, back-propagates through the
compositing and the projection, and updates both parameter sets with one fused
Adam launch.  Every `convert_every` steps the 4D Gaussians whose time scale
exceeds tau become 3D (Sec. 4.1-4.2; the paper classifies at every
densification stage, every 100 iterations), moving their optimizer state along.

Parameters live twice: FP32 master values (and Adam's moments) that the
optimizer updates, and the storage copy the rasterizer reads (BF16, FP16 or the
FP32 master itself), written by the same Adam launch.  The 3D arrays are
allocated for all N Gaussians so the conversion appends in place.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Dict, Optional, Sequence

import torch

from . import abi
from .raster import FIELDS3, FIELDS4, SHAPES, Gaussians, Rasterizer, _ptr, _stream

# step sizes of the 3DGS / 4DGS recipe the paper trains with (positions scaled
# by a scene extent of 5; SH of degree >= 1 at 1/20 of the DC step)
DEFAULT_LR3 = {"mean3": 8e-4, "log_scale3": 5e-3, "quat3": 1e-3, "opacity3": 5e-2, "sh3": 2.5e-3}
DEFAULT_LR4 = {"mean4": 8e-4, "log_scale4": 5e-3, "ql": 1e-3, "qr": 1e-3, "opacity4": 5e-2, "sh4": 2.5e-3}
DEFAULT_LR_SH_REST = 2.5e-3 / 20


class AdamState:
    """Adam's moments for one parameter set (FP32, shaped like the master arrays)."""

    def __init__(self, master: Gaussians, fields: Sequence[str]):
        self.fields = tuple(fields)
        self.m = {k: torch.zeros_like(master.t[k]) for k in self.fields}
        self.v = {k: torch.zeros_like(master.t[k]) for k in self.fields}
        self.c = abi.splat_adam_set()
        for i, k in enumerate(self.fields):
            self.c.param[i] = master.t[k].data_ptr()
            self.c.m[i] = self.m[k].data_ptr()
            self.c.v[i] = self.v[k].data_ptr()


# densification rules of 3DGS that the paper adopts (Sec. 4.3): gradient
# threshold 2e-4 in normalised device coordinates, clones up to 1% of a scene
# extent of 5, split children at 1/1.6 of the scale, pruning below opacity 0.005
DEFAULT_DENSIFY = {"grad_threshold": 2e-4, "dense_scale": 0.05, "min_opacity": 5e-3, "split_shrink": math.log(1.6)}


class Trainer:
    """Batched training of one hybrid scene.  `views` fixes the batch size and
    resolutions; each step may bring other cameras and timestamps.  With
    densify_every > 0 the sets are densified and pruned every densify_every
    steps up to densify_until (before that step's conversion); capacity3 /
    capacity4 bound the sets' rows (default: room for every Gaussian in either
    set, and twice that with densification)."""

    def __init__(self, scene, views: Sequence, dtype=torch.bfloat16, device="cuda", tau: float = 1.0,
                 convert_every: int = 100, lr3: Optional[Dict[str, float]] = None,
                 lr4: Optional[Dict[str, float]] = None, lr_sh_rest: float = DEFAULT_LR_SH_REST,
                 betas=(0.9, 0.999), eps: float = 1e-15, headroom: float = 1.25, densify_every: int = 0,
                 densify_until: int = 15000, densify: Optional[Dict[str, float]] = None,
                 capacity3: Optional[int] = None, capacity4: Optional[int] = None):
        n = scene.n3 + scene.n4
        grow = 2 if densify_every > 0 else 1
        cap3 = capacity3 or grow * n
        cap4 = capacity4 or (grow * n if densify_every > 0 else scene.n4)
        self.master = Gaussians.from_scene(scene, device, dtype=torch.float32, capacity3=cap3, capacity4=cap4)
        self.store = self.master if dtype == torch.float32 else Gaussians.from_scene(scene, device, dtype=dtype,
                                                                                  capacity3=cap3,
                                                                                  capacity4=cap4)
        self.s3 = AdamState(self.master, FIELDS3)
        self.s4 = AdamState(self.master, FIELDS4)
        self.R = Rasterizer(self.master.n3, self.master.n4, views, device=device, keep_keys=False, headroom=headroom,
                            sh_time=self.master.sh_time)
        self.R.autotune_capacity(self.store)
        self.tau = float(tau)
        self.convert_every = int(convert_every)
        self.t = 0
        lr3 = dict(DEFAULT_LR3, **(lr3 or {}))
        lr4 = dict(DEFAULT_LR4, **(lr4 or {}))
        self.hyper = abi.splat_adam_hyper()
        for i, k in enumerate(FIELDS3):
            self.hyper.lr3[i] = lr3[k]
        for i, k in enumerate(FIELDS4):
            self.hyper.lr4[i] = lr4[k]
        self.hyper.lr_sh_rest = lr_sh_rest
        self.hyper.beta1, self.hyper.beta2 = betas
        self.hyper.eps = eps
        dev = self.master.t["mean3"].device
        wb = max(abi.splat_workspace_size_4d(op, self.master.n4, self.master.sh_time)
                 for op in (abi.SPLAT_OP_CONVERT_STATE, abi.SPLAT_OP_CONVERT))
        self.conv_ws = torch.empty((int(wb),), dtype=torch.uint8, device=dev)
        self.n_moved = torch.zeros((1,), dtype=torch.int64, device=dev)
        self.moved_total = 0
        self.views = list(views)
        self.headroom = headroom
        self.densify_every, self.densify_until = int(densify_every), int(densify_until)
        self.rule = abi.splat_densify_rule()
        for k, v in dict(DEFAULT_DENSIFY, **(densify or {})).items():
            setattr(self.rule, k, v)
        if self.densify_every > 0:
            rows = self.master.capacity3 + self.master.capacity4
            self.accum = torch.zeros((rows,), dtype=torch.float32, device=dev)
            self.count = torch.zeros((rows,), dtype=torch.float32, device=dev)
            self.n_out = torch.zeros((2,), dtype=torch.int64, device=dev)

    @property
    def n3(self) -> int:
        return self.master.n3

    @property
    def n4(self) -> int:
        return self.master.n4

    def adam(self, stream=None):
        """The fused Adam launch over both sets (asynchronous)."""
        self.t += 1
        self.hyper.step = self.t
        g3, g4 = self.store.c_g3(), self.store.c_g4()
        abi.check(abi.splat_adam_step(C.byref(self.hyper), C.byref(self.s3.c), C.byref(self.R.cg3), C.byref(g3),
                                      C.byref(self.s4.c), C.byref(self.R.cg4), C.byref(g4), _ptr(self.R.status),
                                      _stream(stream)), "splat_adam_step")

    def step(self, views: Sequence, target: torch.Tensor, stream=None, marks: Optional[dict] = None):
        """Render, loss, backward and update for one batch (asynchronous except at a
        conversion step, which reads the moved count)."""
        self.R.set_views(views)
        self.R.step(self.store, target, stream, marks)
        densifying = self.densify_every > 0 and self.t < self.densify_until
        if densifying:
            abi.check(abi.splat_densify_stats(C.byref(self.R.cproj), self.R.cviews, self.R.V, _ptr(self.R.dproj),
                                              _ptr(self.accum), _ptr(self.count), _stream(stream)),
                      "splat_densify_stats")
        self.adam(stream)
        if densifying and self.t % self.densify_every == 0:
            self.densify(stream)
        if self.convert_every > 0 and self.t % self.convert_every == 0:
            self.convert(stream)

    def convert(self, stream=None) -> int:
        """Sec. 4.1-4.2 with the optimizer state: moments first (the decision reads the
        4D time scales before the conversion rewrites them), then the master
        parameters, then the storage copy.  Synchronises once; returns the count."""
        m3, m4 = self.master.c_g3(), self.master.c_g4()
        st = _stream(stream)
        need = max(abi.splat_workspace_size_4d(op, self.master.n4, self.master.sh_time)
                   for op in (abi.SPLAT_OP_CONVERT_STATE, abi.SPLAT_OP_CONVERT))
        if need > self.conv_ws.numel():  # the 4D set grew by densification
            self.conv_ws = torch.empty((int(need),), dtype=torch.uint8, device=self.conv_ws.device)
        ws, wb = _ptr(self.conv_ws), self.conv_ws.numel()
        abi.check(abi.splat_convert_adam_state(C.byref(m4), C.byref(m3), self.tau, C.byref(self.s4.c),
                                               C.byref(self.s3.c), _ptr(self.R.status), ws, wb, st),
                  "splat_convert_adam_state")
        abi.check(abi.splat_convert_4d_to_3d(C.byref(m4), C.byref(m3), self.tau, _ptr(self.n_moved),
                                             _ptr(self.R.status), ws, wb, st), "splat_convert_4d_to_3d")
        self.R.check("conversion")
        moved = int(self.n_moved.item())
        for G in {id(self.master): self.master, id(self.store): self.store}.values():
            G.n3 += moved
            G.n4 -= moved
        if self.store is not self.master:
            s3, s4 = self.master.c_g3(), self.master.c_g4()
            d3, d4 = self.store.c_g3(), self.store.c_g4()
            abi.check(abi.splat_cast_params(C.byref(s3), C.byref(d3), C.byref(s4), C.byref(d4), st),
                      "splat_cast_params")
        self.R.set_counts(self.master.n3, self.master.n4)
        self.moved_total += moved
        return moved

    def densify(self, stream=None) -> tuple:
        """Clone / split / prune both sets (Sec. 4.3) from the statistics gathered since
        the last call, then the storage copy and a rasterizer for the new counts.
        Synchronises once; returns the new (n3, n4)."""
        n3, n4 = self.master.n3, self.master.n4
        dev = self.accum.device
        noise3 = torch.randn((max(1, n3), 2, 3), device=dev)
        noise4 = torch.randn((max(1, n4), 2, 4), device=dev)
        a, c = self.accum.data_ptr(), self.count.data_ptr()
        d3 = abi.splat_densify_set(n3, self.master.capacity3, C.pointer(self.s3.c), a + 4 * n4, c + 4 * n4,
                                   noise3.data_ptr(), 0)
        d4 = abi.splat_densify_set(n4, self.master.capacity4, C.pointer(self.s4.c), a, c, noise4.data_ptr(),
                                   self.master.sh_time)
        wb = abi.splat_densify_workspace_size(n3, self.master.capacity3, n4, self.master.capacity4,
                                              self.master.sh_time)
        ws = torch.empty((wb,), dtype=torch.uint8, device=dev)
        st = _stream(stream)
        abi.check(abi.splat_densify(C.byref(self.rule), C.byref(d3), C.byref(d4), _ptr(self.n_out),
                                    _ptr(self.R.status), _ptr(ws), wb, st), "splat_densify")
        self.R.check("densification")
        n3, n4 = (int(x) for x in self.n_out.tolist())
        for G in {id(self.master): self.master, id(self.store): self.store}.values():
            G.n3, G.n4 = n3, n4
        if self.store is not self.master:
            s3, s4 = self.master.c_g3(), self.master.c_g4()
            t3, t4 = self.store.c_g3(), self.store.c_g4()
            abi.check(abi.splat_cast_params(C.byref(s3), C.byref(t3), C.byref(s4), C.byref(t4), st),
                      "splat_cast_params")
        self.accum.zero_()
        self.count.zero_()
        cap = self.R.capacity
        self.R = Rasterizer(n3, n4, self.views, device=dev, keep_keys=False, headroom=self.headroom,
                            capacity=cap, sh_time=self.master.sh_time)
        self.R.autotune_capacity(self.store)
        return n3, n4

    def state_dict(self) -> dict:
        """Everything a resumed run needs: the step count, the set sizes, the FP32
        master values and Adam's moments (rows in use only); torch.save-able."""
        n3, n4 = self.master.n3, self.master.n4
        rows = lambda k: n3 if k in FIELDS3 else n4  # noqa: E731
        return {"t": self.t, "n3": n3, "n4": n4, "sh_time": self.master.sh_time,
                "params": {k: self.master.t[k][: rows(k)].clone() for k in FIELDS3 + FIELDS4},
                "m": {k: (self.s3 if k in FIELDS3 else self.s4).m[k][: rows(k)].clone() for k in FIELDS3 + FIELDS4},
                "v": {k: (self.s3 if k in FIELDS3 else self.s4).v[k][: rows(k)].clone() for k in FIELDS3 + FIELDS4}}

    def load_state_dict(self, sd: dict, stream=None):
        """Resume from state_dict(): same N, views and capacities as the saved run."""
        if sd["n3"] + sd["n4"] != self.R.N or sd["sh_time"] != self.master.sh_time:
            raise ValueError("checkpoint of a different scene size or colour model")
        if sd["n3"] > self.master.capacity3 or sd["n4"] > self.master.capacity4:
            raise ValueError("checkpoint larger than this trainer's capacities")
        n3, n4 = sd["n3"], sd["n4"]
        for k in FIELDS3 + FIELDS4:
            n = n3 if k in FIELDS3 else n4
            st = self.s3 if k in FIELDS3 else self.s4
            self.master.t[k][:n].copy_(sd["params"][k])
            st.m[k][:n].copy_(sd["m"][k])
            st.v[k][:n].copy_(sd["v"][k])
        for G in {id(self.master): self.master, id(self.store): self.store}.values():
            G.n3, G.n4 = n3, n4
        if self.store is not self.master:
            s3, s4 = self.master.c_g3(), self.master.c_g4()
            d3, d4 = self.store.c_g3(), self.store.c_g4()
            abi.check(abi.splat_cast_params(C.byref(s3), C.byref(d3), C.byref(s4), C.byref(d4), _stream(stream)),
                      "splat_cast_params")
        self.R.set_counts(n3, n4)
        self.t = int(sd["t"])

    @property
    def loss(self) -> torch.Tensor:
        return self.R.loss
