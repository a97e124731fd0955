"""Full-size workloads through the CUDA graph that the bench replays, against the
FP64 oracle on sampled outputs.

Each case builds the workload, autotunes it, captures one training step
(slice/project, bin/sort, composite, L1 loss, both adjoints) as a CUDA graph and
replays it:
- the rendered pixels at a seeded sample of every view are compared with the
  oracle (run on the stored parameter values) at those pixels;
- the gradients of that same graph are compared with the oracle's for a loss on
  the sampled pixels only.  The L1 loss kernel's gradient is sign(C - target) / n
  with sign(0) = 0, so a target equal to the rendered image everywhere except at
  the sampled pixels (where it is moved by -+0.25) makes the graph's own loss a
  loss on those pixels, with no change to the captured step.

The cases: the video workload the bench times (300k Gaussians, 4 views at
1352x1014 in one batch, BF16 storage); a 500k-Gaussian arc of 8 cameras at mixed
resolutions (1352x1014 and 676x507, FP32); 1M Gaussians at 2704x2028 over 4
views with BF16 and FP16 storage, whose error against the oracle on the original
FP32 values (the storage rounding) is reported beside the parity numbers.  With
SPLAT_PARITY_REPORT set, every case appends its errors as one JSON line there.
"""
import json
import os

import numpy as np
import pytest
import torch

import bench
import oracle as O
from paper_2505_13215_gb300 import abi, autotune, raster, scenes

from parity_util import (GRAD_RTOL, RGB_TOL, fragile_bound, fragile_pixels, grad_fragile_gaussians, grad_fragile_pixels,
                         report,
                         rel_l2)

pytestmark = pytest.mark.gpu

F3 = raster.FIELDS3
F4 = raster.FIELDS4


def _report(name, rec, bench_name=None):
    """Prints and records the measurement; with SPLAT_PRECISION_DIGEST set, also
    files it under the bench's name of the workload in that JSON digest (the
    errors bench.py attaches to its workload entries)."""
    report(name, **rec)
    path = os.environ.get("SPLAT_PRECISION_DIGEST")
    if path and bench_name:
        try:
            with open(path) as fh:
                d = json.load(fh)
        except (OSError, ValueError):
            d = {}
        d.setdefault("how", "tests/test_gpu_workloads.py: the workload's graphed step against the FP64 oracle at "
                            "seeded sample pixels of every view (RGB max-abs over the pixels unique at FP32) and "
                            "the gradients of a loss on those pixels (rel-L2 per tensor); half storage also "
                            "against the oracle on the FP32 originals")
        d.setdefault("workloads", {})[bench_name] = rec
        with open(path, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)


@pytest.fixture(autouse=True)
def _restore_launch_shape():
    yield
    abi.splat_set_pixels_per_lane(8, 8)


def graph_parity(name, scene, views, dtype, n_pix, seed, quant_ref=False, bench_name=None):
    G = raster.Gaussians.from_scene(scene, "cuda", dtype=dtype)
    R = raster.Rasterizer(G.n3, G.n4, views, keep_keys=False)
    target = torch.zeros_like(R.rgb)
    tune = autotune.tune(R, G, target)
    gs = raster.GraphedStep(R, G, target)
    gs.replay()
    torch.cuda.synchronize()
    R.check("graph replay")
    img = R.rgb.clone()
    deq = G.dequantised() if dtype != torch.float32 else scene  # the oracle sees the stored values

    rng = np.random.default_rng(seed)
    n_all = R.rgb.numel()
    dls, Ps, per_view = [], [], []
    target.copy_(img)
    for v, view in enumerate(views):
        npx = view.W * view.H
        pix = np.sort(rng.choice(npx, size=min(n_pix, npx), replace=False))
        P = O.project(deq, view)
        ref = O.render(deq, view, pixels=pix)
        frag = fragile_pixels(P, ref, view, pix)
        got = R.image(v, img).cpu().numpy().reshape(3, -1)[:, pix].astype(np.float64)
        err = np.abs(got - ref["rgb"])[:, ~frag]
        rec = {"view": v, "W": view.W, "H": view.H, "pixels": int(len(pix)), "fragile": int(frag.sum()),
               "rgb_maxabs": float(err.max()) if err.size else 0.0}
        if quant_ref:
            ref32 = O.render(scene, view, pixels=pix)
            rec["rgb_maxabs_vs_fp32_params"] = float(np.abs(got - ref32["rgb"]).max())
        per_view.append(rec)
        assert frag.sum() <= fragile_bound(len(pix), "dense"), rec
        assert rec["rgb_maxabs"] <= RGB_TOL, rec
        # loss on the sampled pixels whose value and gradient are unique at FP32
        sel = pix[~frag & ~grad_fragile_pixels(ref)]
        s = rng.choice([-1.0, 1.0], size=(3, len(sel)))
        tv = R.image(v, target).reshape(3, -1)
        tv[:, torch.from_numpy(sel).cuda()] -= torch.from_numpy(0.25 * s).float().cuda()
        g = np.zeros((3, npx))
        g[:, sel] = s / n_all
        dls.append(g.reshape(3, view.H, view.W))
        Ps.append(P)
    torch.cuda.synchronize()

    gs.replay()
    torch.cuda.synchronize()
    R.check("graph replay with the sampled loss")
    assert torch.equal(img, R.rgb), "the forward of the replay changed"
    nz = int((R.dL != 0).sum().item())
    assert nz == sum(int((np.asarray(d) != 0).sum()) for d in dls)

    tot = None
    for view, g in zip(views, dls):
        r = O.render_bwd(deq, view, g)
        r.pop("dproj")
        tot = r if tot is None else {k: tot[k] + r[k] for k in tot}
    bad = np.zeros(R.N, bool)
    for P in Ps:
        bad |= grad_fragile_gaussians(P)
    bad4, bad3 = bad[: R.n4], bad[R.n4:]
    grads = {}
    for k in F3 + F4:
        a = R.grads[k].cpu().numpy().astype(np.float64)
        keep = ~(bad3 if k in F3 else bad4)
        if keep.sum():
            grads[k] = rel_l2(a[keep], tot[k][keep])
    rec = {"dtype": str(dtype).replace("torch.", ""), "instances": R.instances(),
           "ppl": [tune["ppl_fwd"], tune["ppl_bwd"]], "views": per_view, "grad_rel_l2": grads}
    if quant_ref:
        # the error of the storage rounding itself: the same loss against the
        # oracle on the FP32 originals (a statement, not a tolerance)
        tot32 = None
        for view, g in zip(views, dls):
            r = O.render_bwd(scene, view, g)
            r.pop("dproj")
            tot32 = r if tot32 is None else {k: tot32[k] + r[k] for k in tot32}
        rec["grad_rel_l2_vs_fp32_params"] = {
            k: rel_l2(R.grads[k].cpu().numpy().astype(np.float64)[~(bad3 if k in F3 else bad4)],
                      tot32[k][~(bad3 if k in F3 else bad4)]) for k in grads}
    _report(name, rec, bench_name)
    for k, e in grads.items():
        assert e <= GRAD_RTOL, "%s rel-L2 %.3g (all: %s)" % (k, e, grads)


def test_bench_workload_in_its_graph():
    """300k Gaussians, 4 jittered views at 1352x1014 in one batch, BF16 storage:
    the step and launch shape bench.py times."""
    scene, base = scenes.video_scene(seed=1, n3=bench.N3, n4=bench.N4, W=bench.W, H=bench.H)
    views = scenes.jittered_views(base[0], 4, seed=bench.rank_seed(0))
    graph_parity("video 300k, 4 views 1352x1014, bf16", scene, views, torch.bfloat16, n_pix=400, seed=11,
                 quant_ref=True, bench_name="headline")


def test_arc_500k_eight_mixed_views_fp32():
    scene, views = scenes.arc_scene(seed=2, n=500_000, frac4=0.3, n_views=8)
    graph_parity("arc 500k, 8 views 1352x1014 / 676x507, fp32", scene, views, torch.float32, n_pix=200,
                 seed=12, bench_name=bench.WORKLOADS[0][0])


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_1m_gaussians_4k_four_views_half_storage(dtype):
    full = (2704, 2028, 2920.0)
    scene, views = scenes.arc_scene(seed=3, n=1_000_000, frac4=0.4, n_views=4, full=full, half=full)
    graph_parity("arc 1M, 4 views 2704x2028, %s" % str(dtype).replace("torch.", ""), scene, views, dtype,
                 n_pix=200, seed=13, quant_ref=True,
                 bench_name=bench.WORKLOADS[1 if dtype == torch.bfloat16 else 2][0])
