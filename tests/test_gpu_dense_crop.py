"""Full-resolution parity of the shortened tile lists against the oracle.

With footprint culling and the saturation cut (the defaults), a tile's list
ends once alpha lower bounds certify that every pixel of the tile has
stopped its walk (T below 1e-4); the saturation head takes each 8x8-tile
super-tile's list in order up to HEAD_REACH entries, and tiles still open then
continue, uncut, in tail segments of TAIL_SEG entries.  Here the kernels'
images are compared with the FP64 oracle -- which walks the plain rectangle
lists and knows nothing of the cut -- on EVERY pixel of two 128x128 crops of
the 1352x1014, 300k-Gaussian video workload, through the C ABI:

  - the densest super-tile of the base camera, whose list is longer than the
    head's reach and all of whose tiles end in the head;
  - a super-tile of a turned camera where some tiles end in the head while
    others continue into the tail, with a list long enough to cross a tail
    segment boundary.

Per pixel: RGB within 2e-4, final T within 1e-4 relative, and the Gaussian at
which the walk stops (the entry that would take T below 1e-4, or none) the
same on both sides; then per-tensor gradients of a loss on the crops' pixels
within 1e-3 relative L2.  Pixels whose result is not unique at FP32 are set
aside and counted (the count is in every failure message).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_13215_gb300 import raster, scenes

from parity_util import (GRAD_RTOL, RGB_TOL, fragile_bound, fragile_pixels, grad_fragile_gaussians, grad_fragile_pixels,
                         rel_l2, report)

pytestmark = pytest.mark.gpu

HEAD_REACH = 512   # entries of a super-tile list the saturation head takes in order
TAIL_SEG = 1024    # entries of one tail segment
SUPER = 8          # tiles per super-tile side


def super_list_lengths(R, v):
    """Entries of every super-tile list of view v: the visible rows whose tile
    rectangle, widened to super-tiles, covers it (the level-1 lists the sort
    partitions the depth-ordered rows into)."""
    N = R.N
    rect = R.rect[v * N:(v + 1) * N].cpu().numpy().astype(np.int64)
    vis = R.n_tiles[v * N:(v + 1) * N].cpu().numpy() > 0
    TX, TY = (R.W[v] + 15) // 16, (R.H[v] + 15) // 16
    STX, STY = (TX + SUPER - 1) // SUPER, (TY + SUPER - 1) // SUPER
    r = rect[vis]
    x0, y0 = r[:, 0] // SUPER, r[:, 1] // SUPER
    x1, y1 = (r[:, 2] + SUPER - 1) // SUPER, (r[:, 3] + SUPER - 1) // SUPER
    diff = np.zeros((STY + 1, STX + 1), np.int64)
    np.add.at(diff, (y0, x0), 1)
    np.add.at(diff, (y0, x1), -1)
    np.add.at(diff, (y1, x0), -1)
    np.add.at(diff, (y1, x1), 1)
    return diff.cumsum(0).cumsum(1)[:STY, :STX]


def tile_state(R, v):
    """Per tile of view v: (list start, list length, every pixel's walk ended
    before the list end)."""
    TX, TY = (R.W[v] + 15) // 16, (R.H[v] + 15) // 16
    tb = sum(((w + 15) // 16) * ((h + 15) // 16) for w, h in zip(R.W[:v], R.H[:v]))
    rg = R.ranges.view(-1, 2).cpu().numpy().astype(np.int64)[tb:tb + TX * TY]
    start, length = rg[:, 0].reshape(TY, TX), (rg[:, 1] - rg[:, 0]).reshape(TY, TX)
    last = R.plane(v, R.last).cpu().numpy().astype(np.int64)
    ys, xs = np.mgrid[0:R.H[v], 0:R.W[v]]
    ended = last < length[ys // 16, xs // 16]
    sat = np.ones((TY, TX), bool)
    np.logical_and.at(sat, (ys // 16, xs // 16), ended)
    return start, length, sat


def crop_pixels(view, sx, sy):
    ys, xs = np.mgrid[sy * 128:(sy + 1) * 128, sx * 128:(sx + 1) * 128]
    return (ys * view.W + xs).ravel()


@pytest.fixture(scope="module")
def dense():
    scene, base = scenes.video_scene()
    views = scenes.jittered_views(base[0], 2, seed=100)
    G = raster.Gaussians.from_scene(scene, "cuda")
    R = raster.Rasterizer(G.n3, G.n4, views)
    R.autotune_capacity(G)
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    crops = []
    for v, view in enumerate(views):
        L = super_list_lengths(R, v)
        start, length, sat = tile_state(R, v)
        full_x, full_y = view.W // (16 * SUPER), view.H // (16 * SUPER)  # super-tiles inside the image
        best = None
        for sy in range(full_y):
            for sx in range(full_x):
                blk = (slice(sy * SUPER, (sy + 1) * SUPER), slice(sx * SUPER, (sx + 1) * SUPER))
                s, n = sat[blk], length[blk]
                if v == 0:
                    ok = L[sy, sx] > HEAD_REACH and s.all()
                    score = L[sy, sx]
                else:
                    ok = L[sy, sx] > HEAD_REACH + TAIL_SEG and s.any() and (~s & (n > 0)).any()
                    score = int((~s & (n > 0)).sum())
                if ok and (best is None or score > best[0]):
                    best = (score, sx, sy)
        assert best is not None, "view %d: no super-tile of the kind this test needs" % v
        _, sx, sy = best
        blk = (slice(sy * SUPER, (sy + 1) * SUPER), slice(sx * SUPER, (sx + 1) * SUPER))
        crops.append({"sx": sx, "sy": sy, "list": int(L[sy, sx]), "saturated": int(sat[blk].sum()),
                      "pix": crop_pixels(view, sx, sy)})
    return scene, views, G, R, crops


def test_dense_crops_pixel_for_pixel(dense):
    scene, views, G, R, crops = dense
    K = R.instances()
    vals = R.vals[:K].cpu().numpy().astype(np.int64)
    for v, (view, c) in enumerate(zip(views, crops)):
        pix = c["pix"]
        P = O.project(scene, view)
        ref = O.render(scene, view, pixels=pix)
        frag = fragile_pixels(P, ref, view, pix)
        rec = "view %d super-tile (%d, %d), list %d, %d/64 tiles end in the head, fragile %d/%d" % (
            v, c["sx"], c["sy"], c["list"], c["saturated"], int(frag.sum()), len(pix))
        report("dense crop", view=v, super_tile=[c["sx"], c["sy"]], super_list=c["list"],
               tiles_ending_in_head=c["saturated"], pixels=len(pix), fragile=int(frag.sum()))
        assert frag.sum() <= fragile_bound(len(pix), "dense"), rec
        img = R.image(v).cpu().numpy().reshape(3, -1)[:, pix].astype(np.float64)
        err = np.abs(img - ref["rgb"])[:, ~frag]
        assert err.max() <= RGB_TOL, "rgb max-abs %.3g; %s" % (err.max(), rec)
        T = R.plane(v, R.final_T).cpu().numpy().reshape(-1)[pix]
        np.testing.assert_allclose(T[~frag], ref["T"][~frag], rtol=1e-4, atol=1e-6, err_msg=rec)
        # the Gaussian at which each walk stops (-1: the walk reached its list end)
        start, length, _ = tile_state(R, v)
        last = R.plane(v, R.last).cpu().numpy().reshape(-1)[pix].astype(np.int64)
        u, y = pix % view.W, pix // view.W
        st, ln = start[y // 16, u // 16], length[y // 16, u // 16]
        gpu_stop = np.where(last < ln, vals[np.where(last < ln, st + last, 0)] % R.N, -1)
        lists = {}
        for tx, ty in set(zip((u // 16).tolist(), (y // 16).tolist())):
            lists[(tx, ty)] = O.tile_list(scene, view, tx, ty)
        ora_stop = np.array([lists[(a // 16, b // 16)][l] if l < len(lists[(a // 16, b // 16)]) else -1
                             for a, b, l in zip(u, y, ref["last"])], np.int64)
        bad = (gpu_stop != ora_stop) & ~frag
        assert not bad.any(), "%d walks stop at another Gaussian; %s" % (int(bad.sum()), rec)
        assert (gpu_stop[~frag] >= 0).any(), rec


def test_dense_crops_gradients(dense):
    scene, views, G, R, crops = dense
    rng = np.random.default_rng(17)
    dls, Ps = [], []
    for view, c in zip(views, crops):
        pix = c["pix"]
        P = O.project(scene, view)
        ref = O.render(scene, view, pixels=pix)
        sel = pix[~fragile_pixels(P, ref, view, pix) & ~grad_fragile_pixels(ref)]
        g = np.zeros((3, view.W * view.H))
        g[:, sel] = rng.choice([-1.0, 1.0], size=(3, len(sel))) * 1e-2
        dls.append(g.reshape(3, view.H, view.W))
        Ps.append(P)
    dl = torch.from_numpy(np.concatenate([g.reshape(-1) for g in dls]).astype(np.float32)).cuda()
    R.backward(G, dl)
    torch.cuda.synchronize()
    R.check()
    tot = None
    for view, g in zip(views, dls):
        r = O.render_bwd(scene, view, g.astype(np.float32).astype(np.float64))
        r.pop("dproj")
        tot = r if tot is None else {k: tot[k] + r[k] for k in tot}
    bad = np.zeros(R.N, bool)
    for P in Ps:
        bad |= grad_fragile_gaussians(P)
    bad4, bad3 = bad[:R.n4], bad[R.n4:]
    errs = {}
    for k in raster.FIELDS3 + raster.FIELDS4:
        keep = ~(bad3 if k in raster.FIELDS3 else bad4)
        a = R.grads[k].cpu().numpy().astype(np.float64)[keep]
        b = tot[k][keep]
        if np.linalg.norm(b) > 0:
            errs[k] = rel_l2(a, b)
    assert errs and max(errs.values()) <= GRAD_RTOL, errs
