"""The saturation cut of the binned tile sort, pinned on the FP64 oracle.

Each tile list may end once lower bounds of the entries' alpha over the tile
certify that every pixel of the tile has stopped its walk (Alg. 1: a pixel
stops before the entry that would take T below 1e-4).  Here the bound is
evaluated in FP64 on the oracle's projection -- alpha_lb = alpha_max
exp(-q/2), q the largest quadratic form over the tile's corners clipped to the
image, counted when alpha_lb >= 1.002/255 and a c - b^2 >= 1e-3 a c -- and its
running sum of -ln(1 - alpha_lb) over each tile's depth-ordered list is
compared with where the oracle's own walks end: at every pixel of a tile the
walk must end at or before the entry that takes the sum past 9.25.  Dense
crop of the 300k video view, where the cut engages in most tiles.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2505_13215_gb300 import scenes

THRESHOLD = 9.25  # -ln(1e-4) = 9.2103 plus the margin the kernels use
TILE = 16


def alpha_lower_bound(P, i, x0, x1, y0, y1):
    a, b, c = P["conic"][i]
    if not (a > 0 and c > 0 and a * c - b * b >= 1e-3 * a * c):
        return 0.0
    q = max(a * dx * dx + 2 * b * dx * dy + c * dy * dy
            for dx in (P["px"][i] - x0, P["px"][i] - x1) for dy in (P["py"][i] - y0, P["py"][i] - y1))
    alpha = min(P["alpha"][i] * np.exp(-0.5 * q), 0.98999)
    return alpha if alpha >= 1.002 / 255 else 0.0


@pytest.fixture(scope="module")
def crop():
    scene, base = scenes.video_scene(seed=1)
    v = base[0]
    view = dataclasses.replace(v, W=160, H=128, cx=v.cx - 400.0, cy=v.cy - 300.0)
    return scene, view, O.project(scene, view), O.render(scene, view)


def test_walks_end_before_the_saturation_cut(crop):
    scene, view, P, ref = crop
    W, H = view.W, view.H
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    last = ref["last"].reshape(H, W)
    cut_tiles = 0
    for ty in range(TY):
        for tx in range(TX):
            ids = O.tile_list(scene, view, tx, ty)
            x0, y0 = TILE * tx, TILE * ty
            x1, y1 = min(x0 + TILE - 1, W - 1), min(y0 + TILE - 1, H - 1)
            s = 0.0
            cut = None
            for j, i in enumerate(ids):
                al = alpha_lower_bound(P, i, x0, x1, y0, y1)
                if al > 0:
                    s += -np.log1p(-al)
                if s >= THRESHOLD:
                    cut = j
                    break
            if cut is None:
                continue
            cut_tiles += 1
            blk = last[y0:y1 + 1, x0:x1 + 1]
            assert blk.max() <= cut, (tx, ty, int(blk.max()), cut, len(ids))
            # the bound certifies saturation: every pixel stopped (did not reach the list end)
            assert blk.max() < len(ids)
    # the check is not vacuous: the cut engages in most tiles of this dense crop
    assert cut_tiles >= 0.5 * TX * TY, cut_tiles


def test_alpha_lower_bound_holds_at_every_pixel(crop):
    """The corner maximum bounds the alpha of every pixel of the tile (the
    quadratic form is convex), checked pixel by pixel on a sample of (entry,
    tile) pairs with a positive bound."""
    scene, view, P, ref = crop
    rng = np.random.default_rng(5)
    W, H = view.W, view.H
    checked = 0
    for tx, ty in [(0, 0), (3, 2), (6, 5), (9, 7)]:
        ids = O.tile_list(scene, view, tx, ty)
        x0, y0 = TILE * tx, TILE * ty
        x1, y1 = min(x0 + TILE - 1, W - 1), min(y0 + TILE - 1, H - 1)
        xs, ys = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1))
        for i in rng.choice(ids, size=min(200, len(ids)), replace=False):
            al = alpha_lower_bound(P, i, x0, x1, y0, y1)
            if al == 0:
                continue
            a, b, c = P["conic"][i]
            dx, dy = P["px"][i] - xs, P["py"][i] - ys
            alpha = np.minimum(P["alpha"][i] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)), 0.99)
            assert alpha.min() >= al * (1 - 1e-12), (i, tx, ty)
            checked += 1
    assert checked >= 50, checked
