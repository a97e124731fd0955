"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (see parity_util): rendered RGB max-abs 2e-4 on every pixel whose
result is unique at FP32; parameter gradients 1e-3 relative L2 per tensor;
sorted per-tile instance lists bit-exact when both sides sort the same keys.
"""
import ctypes as C
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_13215_gb300 import abi, raster, scenes

from parity_util import (GRAD_RTOL, RGB_TOL, fragile_bound, fragile_gaussians, fragile_pixels, grad_fragile_gaussians,
                         grad_fragile_pixels, rel_l2, report)

pytestmark = pytest.mark.gpu

F3 = raster.FIELDS3
F4 = raster.FIELDS4


class tile_cull:
    """Context: footprint culling of the binned tile lists on / off."""

    def __init__(self, on):
        self.on = on

    def __enter__(self):
        abi.splat_set_tile_cull(self.on)

    def __exit__(self, *exc):
        abi.splat_set_tile_cull(True)


def make(scene, views, dtype=torch.float32, capacity3=None):
    G = raster.Gaussians.from_scene(scene, "cuda", dtype=dtype, capacity3=capacity3)
    R = raster.Rasterizer(G.n3, G.n4, views, sh_time=G.sh_time)
    R.autotune_capacity(G)
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    return G, R


@pytest.fixture(scope="module")
def small():
    scene, views = scenes.small_scene(seed=0)
    G, R = make(scene, views)
    P = O.project(scene, views[0])
    ref = O.render(scene, views[0])
    return scene, views, G, R, P, ref


# ---------------------------------------------------------------------------
# A1-A4: slice + project
# ---------------------------------------------------------------------------

def check_projection(R, P, v=0):
    N = R.N
    sl = slice(v * N, (v + 1) * N)
    rad = R.radius[sl].cpu().numpy()
    rect = R.rect[sl].cpu().numpy()
    nt = R.n_tiles[sl].cpu().numpy()
    xy = R.xy[sl].cpu().numpy().astype(np.float64)
    co = R.conic_opacity[sl].cpu().numpy().astype(np.float64)
    rd = R.rgb_depth[sl].cpu().numpy().astype(np.float64)
    sure = ~fragile_gaussians(P)
    vis_o = P["visible"] == 1
    vis_g = rad > 0
    np.testing.assert_array_equal(vis_g[sure], vis_o[sure])
    np.testing.assert_array_equal(rad[sure & vis_o], P["radius"][sure & vis_o])
    np.testing.assert_array_equal(rect[sure & vis_o], P["rect"][sure & vis_o])
    np.testing.assert_array_equal(nt[sure & vis_o], P["n_tiles"][sure & vis_o])
    both = vis_g & vis_o
    assert both.sum() > 0
    o = P[both]
    np.testing.assert_allclose(xy[both, 0], o["px"], rtol=1e-5, atol=2e-3)
    np.testing.assert_allclose(xy[both, 1], o["py"], rtol=1e-5, atol=2e-3)
    scale = np.maximum(np.abs(o["conic"][:, 0]), np.abs(o["conic"][:, 2]))
    for k in range(3):
        assert np.max(np.abs(co[both, k] - o["conic"][:, k]) / scale) < 1e-4
    np.testing.assert_allclose(co[both, 3], o["alpha"], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(rd[both, :3], o["rgb"], atol=2e-5)
    np.testing.assert_allclose(rd[both, 3], o["depth"], rtol=1e-6)
    return int((~sure).sum())


def test_slice_project_matches_oracle(small):
    scene, views, G, R, P, ref = small
    n_fragile = check_projection(R, P)
    assert n_fragile < 0.01 * R.N


# ---------------------------------------------------------------------------
# A5-A8: bin + sort (staged: both sides sort the same keys)
# ---------------------------------------------------------------------------

def staged_sort(views, proj_per_view, N, depth_override=None):
    """Feed oracle rectangles / float32 depths to splat_bin_sort; return the GPU
    lists and the oracle's stable sort of the same keys."""
    V = len(views)
    abi.splat_set_tile_cull(False)  # the oracle lists every tile of the rectangle
    R = raster.Rasterizer(N, 0, views)
    keys_o, ids_o = [], []
    tile_base = 0
    for v, (view, P) in enumerate(zip(views, proj_per_view)):
        dep = P["depth"].astype(np.float32) if depth_override is None else depth_override[v]
        sl = slice(v * N, (v + 1) * N)
        vis = P["visible"] == 1
        R.rect[sl] = torch.from_numpy(np.where(vis[:, None], P["rect"], 0).astype(np.int32)).cuda()
        R.n_tiles[sl] = torch.from_numpy(np.where(vis, P["n_tiles"], 0).astype(np.int32)).cuda()
        R.radius[sl] = torch.from_numpy(np.where(vis, P["radius"], 0).astype(np.int32)).cuda()
        rd = np.zeros((N, 4), np.float32)
        rd[:, 3] = dep
        R.rgb_depth[sl] = torch.from_numpy(rd).cuda()
        k, ids = O.tile_keys(P, view, depth_f32=dep)
        k = k + (np.uint64(tile_base) << np.uint64(32))
        keys_o.append(k)
        ids_o.append(ids + v * N)
        tile_base += ((view.W + 15) // 16) * ((view.H + 15) // 16)
    keys_o = np.concatenate(keys_o) if keys_o else np.zeros(0, np.uint64)
    ids_o = np.concatenate(ids_o) if ids_o else np.zeros(0, np.int64)
    perm = O.stable_sort_u64(keys_o)
    K = len(keys_o)
    R.set_capacity(K + 100)
    R.status.zero_()
    st = C.c_void_p(R.status.data_ptr())
    abi.check(abi.splat_bin_sort(C.byref(R.cproj), R.cviews, V, C.byref(R.cbins), st, C.c_void_p(R.ws.data_ptr()),
                                 R.ws_bytes, C.c_void_p(torch.cuda.current_stream().cuda_stream)), "bin_sort")
    torch.cuda.synchronize()
    abi.splat_set_tile_cull(True)
    R.check()
    assert R.instances() == K
    gk = R.keys[:K].cpu().numpy().astype(np.uint32)
    gv = R.vals[:K].cpu().numpy().astype(np.uint32)
    ok = (keys_o[perm] >> np.uint64(32)).astype(np.uint32)
    ov = ids_o[perm].astype(np.uint32)
    ranges = R.ranges.cpu().numpy().reshape(-1, 2)
    return gk, gv, ok, ov, ranges, tile_base


def expected_ranges(sorted_tiles, total):
    r = np.zeros((total, 2), np.int64)
    for t in np.unique(sorted_tiles):
        w = np.nonzero(sorted_tiles == t)[0]
        r[t] = (w[0], w[-1] + 1)
    return r


@pytest.fixture(params=[2, 1], ids=["binned", "radix"])
def tile_sort_mode(request):
    abi.splat_set_tile_sort(request.param)
    yield request.param
    abi.splat_set_tile_sort(0)


def test_bin_sort_bitexact_given_keys(small, tile_sort_mode):
    scene, views, G, R, P, ref = small
    gk, gv, ok, ov, ranges, T = staged_sort(views, [P], R.N)
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)
    np.testing.assert_array_equal(ranges, expected_ranges(ok, T))


def test_bin_sort_ties_and_multiview(tile_sort_mode):
    """Equal depths everywhere (ties broken by emission order) over three views of
    different sizes in one call."""
    scene, _ = scenes.small_scene(seed=2, n3=700, n4=300)
    views = [scenes.identity_view(128, 128, 128.0, 0.5), scenes.identity_view(80, 48, 70.0, 0.2),
             scenes.identity_view(200, 120, 150.0, 0.9)]
    Ps = [O.project(scene, v) for v in views]
    rng = np.random.default_rng(3)
    deps = [rng.choice(np.array([2.0, 3.0, 3.0000002, 5.0], np.float32), size=scene.n) for _ in views]
    gk, gv, ok, ov, ranges, T = staged_sort(views, Ps, scene.n, depth_override=deps)
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)
    np.testing.assert_array_equal(ranges, expected_ranges(ok, T))


def test_bin_sort_crowded_depths(tile_sort_mode):
    """Two thirds of 6000 rows per view at one of two depths (as BF16-rounded
    means produce in dense depth ranges): thousands of exact depth ties per
    view, broken in emission order, the lists bit-exact in both tile-sort modes."""
    scene, _ = scenes.small_scene(seed=4, n3=4200, n4=1800)
    views = [scenes.identity_view(160, 128, 150.0, 0.3), scenes.identity_view(96, 80, 90.0, 0.7)]
    Ps = [O.project(scene, v) for v in views]
    rng = np.random.default_rng(5)
    deps = []
    for _ in views:
        d = rng.uniform(1.5, 6.0, scene.n).astype(np.float32)
        crowd = rng.random(scene.n) < 2.0 / 3.0
        d[crowd] = rng.choice(np.array([2.5, 4.0], np.float32), size=int(crowd.sum()))
        deps.append(d)
    gk, gv, ok, ov, ranges, T = staged_sort(views, Ps, scene.n, depth_override=deps)
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)
    np.testing.assert_array_equal(ranges, expected_ranges(ok, T))


def test_bin_sort_bitexact_at_scale(tile_sort_mode):
    """Three views of different sizes (704x528, 512x400, 880x300) of a frustum
    scene of 18k Gaussians at depths 1-20, the near ones covering many tiles:
    several super-tiles per view, super-tile lists of several runs of 4096 slots
    with rows cut across runs, and more tiles than one block of the tile
    ranges takes.  Lists, ranges and K bit-exact against the oracle's stable
    sort of the same keys."""
    import dataclasses
    scene, base = scenes.video_scene(seed=5, n3=12000, n4=6000, W=704, H=528, f=760.0)
    jit = scenes.jittered_views(base[0], 3, seed=11)
    views = [jit[0], dataclasses.replace(jit[1], W=512, H=400, cx=256.0, cy=200.0),
             dataclasses.replace(jit[2], W=880, H=300, cx=440.0, cy=150.0)]
    Ps = [O.project(scene, v) for v in views]
    # the split's work at this size: super-tile entries per view, tiles in all
    for P in Ps:
        r = P["rect"][P["visible"] == 1].astype(np.int64)
        k1 = (((r[:, 2] + 7) >> 3) - (r[:, 0] >> 3)) * (((r[:, 3] + 7) >> 3) - (r[:, 1] >> 3))
        assert k1.sum() > 3 * 4096 and k1.max() >= 16
    gk, gv, ok, ov, ranges, T = staged_sort(views, Ps, scene.n)
    assert T > 2 * 1024
    np.testing.assert_array_equal(gk, ok)
    np.testing.assert_array_equal(gv, ov)
    np.testing.assert_array_equal(ranges, expected_ranges(ok, T))


def test_bin_sort_end_to_end_lists(small):
    """The GPU's own keys: per tile the same Gaussians, in non-decreasing oracle depth."""
    scene, views, G, R0, P, ref = small
    with tile_cull(False):
        R = raster.Rasterizer(G.n3, G.n4, views)
        R.autotune_capacity(G)
        R.forward(G)
        torch.cuda.synchronize()
        R.check()
    K = R.instances()
    gk = R.keys[:K].cpu().numpy()
    gv = R.vals[:K].cpu().numpy()
    ranges = R.ranges.cpu().numpy().reshape(-1, 2)
    fragile = fragile_gaussians(P)
    for t in range(R.total_tiles):
        s, e = ranges[t]
        assert np.all(gk[s:e] == t)
        ids = gv[s:e].astype(np.int64)
        ref_ids = O.tile_list(scene, views[0], t % 8, t // 8)
        a = set(ids[~fragile[ids]].tolist())
        b = set(ref_ids[~fragile[ref_ids]].tolist())
        assert a == b, "tile %d" % t
        d = P["depth"][ids]
        assert np.all(np.diff(d) >= -1e-6 * d[1:])


# ---------------------------------------------------------------------------
# A9: composite forward
# ---------------------------------------------------------------------------

def check_image(R, P, ref, view, v=0, check_last=False):
    """RGB and final T against the oracle on the pixels unique at FP32; `last` (an
    index into the tile list) only when the lists are the oracle's full rectangles.
    The pixels set aside are counted, reported and bounded (fragile_bound)."""
    img = R.image(v).cpu().numpy().reshape(3, -1).astype(np.float64)
    T = R.plane(v, R.final_T).cpu().numpy().reshape(-1)
    last = R.plane(v, R.last).cpu().numpy().reshape(-1)
    frag = fragile_pixels(P, ref, view)
    err = np.abs(img - ref["rgb"])[:, ~frag]
    note = "fragile pixels %d of %d" % (int(frag.sum()), frag.size)
    report(os.environ.get("PYTEST_CURRENT_TEST", "check_image").split(" ")[0], view=v, pixels=int(frag.size),
           fragile=int(frag.sum()), rgb_maxabs=float(err.max()))
    assert frag.sum() <= fragile_bound(frag.size), note
    assert err.max() <= RGB_TOL, "rgb max-abs %.3g; %s" % (err.max(), note)
    if check_last:
        np.testing.assert_array_equal(last[~frag], ref["last"][~frag], err_msg=note)
    np.testing.assert_allclose(T[~frag], ref["T"][~frag], rtol=1e-4, atol=1e-6, err_msg=note)
    return frag.mean(), err.max()


def test_composite_fwd_matches_oracle(small):
    scene, views, G, R, P, ref = small
    frac, err = check_image(R, P, ref, views[0])


def test_composite_fwd_full_rectangles_last_index(small):
    """Without footprint culling the lists are the oracle's, so `last` matches too."""
    scene, views, G, R0, P, ref = small
    with tile_cull(False):
        R = raster.Rasterizer(G.n3, G.n4, views)
        R.autotune_capacity(G)
        R.forward(G)
        torch.cuda.synchronize()
        R.check()
    check_image(R, P, ref, views[0], check_last=True)


def test_footprint_culling_changes_nothing_but_the_lists(small):
    scene, views, G, R0, P, ref = small
    target = torch.rand(R0.rgb.shape, generator=torch.Generator(device="cuda").manual_seed(9), device="cuda")
    out = []
    for on in (False, True):
        with tile_cull(on):
            R = raster.Rasterizer(G.n3, G.n4, views)
            R.autotune_capacity(G)
            R.step(G, target)
            torch.cuda.synchronize()
            R.check()
            out.append((R.instances(), R.rgb.clone(), R.final_T.clone(), {k: v.clone() for k, v in R.grads.items()}))
    (k0, rgb0, T0, g0), (k1, rgb1, T1, g1) = out
    assert k1 < k0
    assert torch.equal(rgb0, rgb1) and torch.equal(T0, T1)
    for k in g0:
        assert rel_l2(g1[k].cpu().numpy(), g0[k].cpu().numpy()) < 1e-5, k


def test_saturation_cut_changes_nothing_but_the_lists():
    """The 300k-Gaussian video scene seen by the base camera and a turned one
    (the bench's camera batch): with culling on, each tile's list ends once the
    alpha lower bounds certify T < 1e-4 at every pixel of the tile -- in the
    base view every super-tile saturates within the head pass, the turned view
    sees sparse regions whose tiles continue in the tail, and some super-tiles
    hold both (the sort's diagnostic counters show it) -- so the lists shrink
    to a fraction of the rectangle lists, while the images, the transmittance
    and the gradients are those of the full lists, and every pixel's walk stops
    at the same Gaussian (or at the end of its list in both runs)."""
    scene, base = scenes.video_scene()
    views = scenes.jittered_views(base[0], 2, seed=100)
    G = raster.Gaussians.from_scene(scene, "cuda")
    n_pix = sum(v.W * v.H for v in views)
    target = torch.rand((3 * n_pix,), generator=torch.Generator(device="cuda").manual_seed(4), device="cuda")

    def stops(R):
        """Per pixel of every view: the row (Gaussian) at which its walk stopped, -1 at the list end."""
        K = R.instances()
        vals = R.vals[:K].cpu().numpy().astype(np.int64)
        rg = R.ranges.view(-1, 2).cpu().numpy().astype(np.int64)
        res, base_t = [], 0
        for v, view in enumerate(views):
            last = R.plane(v, R.last).cpu().numpy().astype(np.int64)
            ys, xs = np.mgrid[0:view.H, 0:view.W]
            TX = (view.W + 15) // 16
            t = base_t + (ys // 16) * TX + xs // 16
            start, length = rg[t, 0], rg[t, 1] - rg[t, 0]
            sat = last < length
            res.append(np.where(sat, vals[np.where(sat, start + last, 0)], -1))
            base_t += TX * ((view.H + 15) // 16)
        return res

    out = []
    counters = torch.zeros(8, dtype=torch.int64, device="cuda")
    for on in (False, True):
        with tile_cull(on):
            R = raster.Rasterizer(G.n3, G.n4, views)
            R.autotune_capacity(G)
            if on:  # the sort's diagnostic counters of the culled step (the images do not change)
                R.set_options(stats=counters.data_ptr())
                counters.zero_()
            R.step(G, target)
            torch.cuda.synchronize()
            R.check()
            out.append((R.instances(), int(R.n_needed.item()), stops(R), R.rgb.clone(), R.final_T.clone(),
                        {k: v.clone() for k, v in R.grads.items()}))
            del R
    (k0, n0, st0, rgb0, T0, g0), (k1, n1, st1, rgb1, T1, g1) = out
    assert k1 < 0.5 * k0, (k0, k1)
    # the case where the head's cut and the tail's 'done' mask both matter: a
    # super-tile some of whose tiles' lists ended in the head while others
    # continued in its tail segments
    c = counters.cpu().numpy()
    assert c[4] > 0 and c[5] > 0, c
    assert n1 >= k1 and n0 == k0
    assert torch.equal(rgb0, rgb1) and torch.equal(T0, T1)
    for k in g0:
        assert rel_l2(g1[k].cpu().numpy(), g0[k].cpu().numpy()) < 1e-5, k
    for v in range(len(views)):
        np.testing.assert_array_equal(st1[v], st0[v], err_msg="view %d" % v)
        assert (st1[v] >= 0).any()


@pytest.mark.parametrize("ppl", [(2, 2), (4, 4), (2, 8), (8, 4)])
def test_composite_pixels_per_lane_variants(small, ppl):
    """Every compositing variant (2, 4 or 8 pixels per lane, a warp per band of
    the tile) against the oracle, forward and gradients, also with different
    variants in the two passes (the backward reads where each pixel's walk
    ended, whatever band shape wrote it)."""
    scene, views, G, R, P, ref = small
    abi.splat_set_pixels_per_lane(*ppl)
    try:
        R.forward(G)
        torch.cuda.synchronize()
        R.check()
        check_image(R, P, ref, views[0])
        dls = loss_grad(R, [ref], [P], views, seed=3)
        check_grads(R, G, scene, [P], views, dls)
    finally:
        abi.splat_set_pixels_per_lane(8, 8)
        R.forward(G)
        torch.cuda.synchronize()


def test_tile_sort_modes_render_identically(small):
    scene, views, G, R0, P, ref = small
    out = []
    for mode in (1, 2):
        abi.splat_set_tile_sort(mode)
        abi.splat_set_tile_cull(False)
        try:
            R = raster.Rasterizer(G.n3, G.n4, views)
            R.autotune_capacity(G)
            target = torch.rand(R.rgb.shape, generator=torch.Generator(device="cuda").manual_seed(5), device="cuda")
            R.step(G, target)
            torch.cuda.synchronize()
            R.check()
            K = R.instances()
            out.append((R.rgb.clone(), R.vals[:K].clone(), R.ranges.clone(), R.grads["mean3"].clone()))
        finally:
            abi.splat_set_tile_sort(0)
            abi.splat_set_tile_cull(True)
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])
    assert rel_l2(out[0][3].cpu().numpy(), out[1][3].cpu().numpy()) < 1e-5


def test_forward_is_deterministic(small):
    scene, views, G, R, P, ref = small
    R.forward(G)
    a = R.rgb.clone()
    k = R.vals[: R.instances()].clone()
    R.forward(G)
    torch.cuda.synchronize()
    assert torch.equal(a, R.rgb)
    assert torch.equal(k, R.vals[: R.instances()])


# ---------------------------------------------------------------------------
# A10 + A11: backward
# ---------------------------------------------------------------------------

def loss_grad(R, refs, Ps, views, seed=0):
    """dL/dC of an L1 loss against a seeded target, from the oracle image, zero at
    pixels whose value or gradient is not unique at FP32."""
    rng = np.random.default_rng(seed)
    out = []
    for v, (ref, P, view) in enumerate(zip(refs, Ps, views)):
        target = rng.uniform(0, 1, ref["rgb"].shape)
        g = np.sign(ref["rgb"] - target) / ref["rgb"].size
        frag = fragile_pixels(P, ref, view) | grad_fragile_pixels(ref)
        g[:, frag] = 0.0
        out.append(g.reshape(3, view.H, view.W))
    return out


def check_grads(R, G, scene, Ps, views, dls, exclude=None):
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
    if exclude is not None:
        bad |= exclude
    bad4, bad3 = bad[: R.n4], bad[R.n4:]
    worst = {}
    for k in F3 + F4:
        a = R.grads[k].cpu().numpy().astype(np.float64)
        b = tot[k]
        keep = ~(bad3 if k in F3 else bad4)
        if keep.sum() == 0:
            continue
        e = rel_l2(a[keep], b[keep])
        worst[k] = e
    for k, e in worst.items():
        assert e <= GRAD_RTOL, "%s rel-L2 %.3g (all: %s)" % (k, e, worst)
    return worst


def test_gradients_match_oracle(small):
    scene, views, G, R, P, ref = small
    dls = loss_grad(R, [ref], [P], views)
    check_grads(R, G, scene, [P], views, dls)


def test_dproj_matches_oracle(small):
    scene, views, G, R, P, ref = small
    dls = loss_grad(R, [ref], [P], views, seed=1)
    dl = torch.from_numpy(dls[0].reshape(-1).astype(np.float32)).cuda()
    R.backward(G, dl, stop_2d=True)
    torch.cuda.synchronize()
    R.check()
    got = R.dproj.view(-1, 12)[:, :9].cpu().numpy().astype(np.float64)
    want = O.render_bwd(scene, views[0], dls[0].astype(np.float32).astype(np.float64))["dproj"]
    for name, cols in (("xy", [0, 1]), ("conic", [2, 3, 4]), ("alpha", [5]), ("rgb", [6, 7, 8])):
        assert rel_l2(got[:, cols], want[:, cols]) <= GRAD_RTOL, name


# ---------------------------------------------------------------------------
# Multi-view batch in one launch per stage, uneven resolutions
# ---------------------------------------------------------------------------

def test_batched_views_match_oracle():
    scene, views = scenes.arc_scene(seed=5, n=20000, frac4=0.3, n_views=3, full=(256, 192, 280.0),
                                    half=(120, 96, 130.0))
    G, R = make(scene, views)
    Ps = [O.project(scene, v) for v in views]
    refs = [O.render(scene, v) for v in views]
    for v in range(3):
        check_projection(R, Ps[v], v)
        check_image(R, Ps[v], refs[v], views[v], v)
    dls = loss_grad(R, refs, Ps, views, seed=4)
    check_grads(R, G, scene, Ps, views, dls)


# ---------------------------------------------------------------------------
# Full size (1352x1014, 200k 3D + 100k 4D), per-view launch: sampled outputs
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    scene, views = scenes.video_scene(seed=1)
    G, R = make(scene, views)
    P = O.project(scene, views[0])
    return scene, views, G, R, P


def test_full_size_projection(big):
    scene, views, G, R, P = big
    n_fragile = check_projection(R, P)
    assert n_fragile < 0.002 * R.N


def test_full_size_sampled_pixels_and_gradients(big):
    scene, views, G, R, P = big
    view = views[0]
    rng = np.random.default_rng(7)
    pix = rng.choice(view.W * view.H, size=600, replace=False)
    ref = O.render(scene, view, pixels=pix)
    img = R.image(0).cpu().numpy().reshape(3, -1)[:, pix]
    frag = fragile_pixels(P, ref, view, pix)
    err = np.abs(img - ref["rgb"])[:, ~frag]
    note = "fragile pixels %d of %d" % (int(frag.sum()), len(pix))
    report("full size sampled", pixels=len(pix), fragile=int(frag.sum()), rgb_maxabs=float(err.max()))
    assert frag.sum() <= fragile_bound(len(pix), "dense"), note
    assert err.max() <= RGB_TOL, "rgb max-abs %.3g; %s" % (err.max(), note)
    # gradient of a loss on the sampled, unique pixels only
    sel = pix[~frag & ~grad_fragile_pixels(ref)]
    g = np.zeros((3, view.W * view.H))
    g[:, sel] = rng.choice([-1.0, 1.0], size=(3, len(sel))) * 1e-2
    check_grads(R, G, scene, [P], views, [g.reshape(3, view.H, view.W)])


# ---------------------------------------------------------------------------
# Storage precision: BF16 / FP16 parameters, FP32 arithmetic
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_half_storage_matches_oracle_on_stored_values(dtype):
    scene, views = scenes.small_scene(seed=6)
    G, R = make(scene, views, dtype=dtype)
    deq = G.dequantised()
    P = O.project(deq, views[0])
    ref = O.render(deq, views[0])
    check_projection(R, P)
    check_image(R, P, ref, views[0])
    dls = loss_grad(R, [ref], [P], views, seed=2)
    check_grads(R, G, deq, [P], views, dls)


# ---------------------------------------------------------------------------
# A12: 4D -> 3D conversion
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_convert_matches_oracle(dtype):
    scene, _ = scenes.small_scene(seed=8, n3=500, n4=1500)
    G = raster.Gaussians.from_scene(scene, "cuda", dtype=dtype, capacity3=scene.n3 + scene.n4)
    deq = G.dequantised()
    tau = 0.15
    moved, app, keep = O.convert(deq, tau)
    n3_0 = G.n3
    m = raster.convert_4d_to_3d(G, tau)
    assert m == int(moved.sum()) and 0 < m < scene.n4
    got3 = {k: G.t[k][n3_0: n3_0 + m].float().cpu().double().numpy() for k in F3}
    for k in ("mean3", "log_scale3", "opacity3", "sh3"):
        np.testing.assert_array_equal(got3[k], app[k])  # copied bit for bit
    qtol = 2e-5 if dtype == torch.float32 else 8e-3
    np.testing.assert_allclose(got3["quat3"], app["quat3"], atol=qtol)
    for k in F4:
        got = G.t[k][: G.n4].float().cpu().double().numpy()
        np.testing.assert_array_equal(got, deq[k][keep])
    # the old 3D rows are untouched
    for k in F3:
        np.testing.assert_array_equal(G.t[k][:n3_0].float().cpu().double().numpy(), deq[k])


def test_convert_capacity_overflow_changes_nothing():
    scene, _ = scenes.small_scene(seed=8, n3=100, n4=400)
    G = raster.Gaussians.from_scene(scene, "cuda", capacity3=110)
    before = {k: G.t[k].clone() for k in F3 + F4}
    with pytest.raises(abi.SplatError) as e:
        raster.convert_4d_to_3d(G, 0.05)
    assert e.value.code == abi.SPLAT_ERR_CAPACITY
    for k in F3 + F4:
        assert torch.equal(before[k], G.t[k])


# ---------------------------------------------------------------------------
# Edge cases and device-side error reporting
# ---------------------------------------------------------------------------

def test_capacity_overflow_is_reported_then_autotuned(small):
    scene, views, G, R0, P, ref = small
    R = raster.Rasterizer(G.n3, G.n4, views, capacity=100)
    R.forward(G)
    code, stage, aux = R.read_status()
    # the needed count, or on the binned path possibly a lower bound of it
    assert code == abi.SPLAT_ERR_CAPACITY and 100 < aux <= R0.instances()
    R.set_capacity(R0.instances())
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    assert R.instances() == R0.instances()
    R.set_capacity(R0.instances() - 1)
    R.forward(G)
    code, stage, aux = R.read_status()
    assert code == abi.SPLAT_ERR_CAPACITY and aux == R0.instances()
    R.autotune_capacity(G)
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    assert torch.equal(R.rgb, R0.rgb)


def test_empty_and_fully_culled_scenes():
    empty = scenes.empty_scene()
    view = scenes.identity_view(40, 24, 40.0, 0.0)
    view.bg = (0.25, 0.5, 1.0)
    G = raster.Gaussians.from_scene(empty, "cuda")
    R = raster.Rasterizer(0, 0, [view])
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    img = R.image(0).cpu().numpy()
    np.testing.assert_array_equal(img, np.broadcast_to(np.array(view.bg, np.float32)[:, None, None], img.shape))
    # everything behind the camera
    scene, _ = scenes.small_scene(seed=1, n3=50, n4=20)
    back = scenes.View(R=np.diag([-1.0, 1.0, -1.0]).astype(np.float32), T=np.zeros(3, np.float32), fx=40.0, fy=40.0,
                       cx=20.0, cy=12.0, W=40, H=24, t=0.5, bg=(0.1, 0.2, 0.3))
    G = raster.Gaussians.from_scene(scene, "cuda")
    R = raster.Rasterizer(G.n3, G.n4, [back])
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    assert R.instances() == 0
    np.testing.assert_allclose(R.image(0).cpu().numpy()[:, 5, 7], [0.1, 0.2, 0.3])
    dl = torch.ones_like(R.rgb)
    R.backward(G, dl)
    torch.cuda.synchronize()
    R.check()
    for k in F3 + F4:
        assert float(R.grads[k].abs().max()) == 0.0


def test_only_3d_and_only_4d():
    for n3, n4 in ((200, 0), (0, 200)):
        scene, views = scenes.small_scene(seed=9, n3=n3, n4=n4)
        G, R = make(scene, views)
        P = O.project(scene, views[0])
        ref = O.render(scene, views[0])
        check_image(R, P, ref, views[0])


def test_spin_limit_zero_reports_or_completes(big):
    scene, views, G, R, P = big
    good = R.rgb.clone()
    abi.splat_set_spin_limit(0)
    try:
        R.forward(G)
        torch.cuda.synchronize()
        code, stage, aux = R.read_status()
        assert code in (abi.SPLAT_OK, abi.SPLAT_ERR_TIMEOUT)
        if code == abi.SPLAT_ERR_TIMEOUT:  # a look-back: depth passes, scan and split, tile ranges, tile passes
            assert abi.STAGES[stage] in ("depth_sort", "scan", "duplicate", "tile_sort")
    finally:
        abi.splat_set_spin_limit(1 << 22)
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    assert torch.equal(good, R.rgb)


def test_invalid_arguments_are_rejected_on_host(small):
    scene, views, G, R, P, ref = small
    st = C.c_void_p(R.status.data_ptr())
    s = C.c_void_p(0)
    g3, g4 = G.c_g3(), G.c_g4()
    assert abi.splat_slice_project(C.byref(g3), C.byref(g4), R.cviews, 0, C.byref(R.cproj), st, s) == abi.SPLAT_ERR_INVALID_ARG
    bad = abi.splat_proj.from_buffer_copy(R.cproj)
    bad.n = R.N + 1
    assert abi.splat_slice_project(C.byref(g3), C.byref(g4), R.cviews, 1, C.byref(bad), st, s) == abi.SPLAT_ERR_INVALID_ARG
    assert abi.splat_bin_sort(C.byref(R.cproj), R.cviews, 1, C.byref(R.cbins), st, C.c_void_p(R.ws.data_ptr()), 16,
                              s) == abi.SPLAT_ERR_INVALID_ARG


def test_l1_loss_kernel(small):
    scene, views, G, R, P, ref = small
    target = torch.rand_like(R.rgb)
    R.l1_loss(target)
    torch.cuda.synchronize()
    d = (R.rgb - target).double()
    assert abs(float(R.loss.item()) - float(d.abs().sum())) < 1e-3 * float(d.abs().sum())
    np.testing.assert_array_equal(R.dL.cpu().numpy(), (torch.sign(d) / R.rgb.numel()).float().cpu().numpy())


@pytest.mark.parametrize("ppl", [4, 8])
def test_forward_with_fused_l1_loss(ppl):
    """splat_composite_fwd_l1 against splat_composite_fwd + splat_l1_loss on a
    3-view batch of mixed sizes: the same image, T and ends of walks, the same
    pixel gradient bit for bit (including sign(0) = 0 where the target equals
    the image), the loss up to the order of its sum."""
    scene, views = scenes.arc_scene(seed=5, n=20000, frac4=0.3, n_views=3, full=(256, 192, 280.0),
                                    half=(120, 96, 130.0))
    G, R = make(scene, views)
    abi.splat_set_pixels_per_lane(ppl, ppl)
    try:
        R.forward(G)
        torch.cuda.synchronize()
        target = torch.rand(R.rgb.shape, generator=torch.Generator(device="cuda").manual_seed(17), device="cuda")
        target[::7] = R.rgb[::7]  # ties: sign(0) = 0
        R.l1_loss(target)
        torch.cuda.synchronize()
        R.check()
        ref = (R.rgb.clone(), R.final_T.clone(), R.last.clone(), R.dL.clone(), float(R.loss.item()))
        R.dL.zero_()
        R.rgb.zero_()
        R.composite_l1(target)
        torch.cuda.synchronize()
        R.check()
    finally:
        abi.splat_set_pixels_per_lane(8, 8)
    assert torch.equal(R.rgb, ref[0]) and torch.equal(R.final_T, ref[1]) and torch.equal(R.last, ref[2])
    assert torch.equal(R.dL, ref[3])
    assert int((R.dL == 0).sum()) >= R.rgb.numel() // 7
    assert abs(float(R.loss.item()) - ref[4]) <= 1e-5 * ref[4]


def test_graph_replay_matches_eager(small):
    scene, views, G, R0, P, ref = small
    R = raster.Rasterizer(G.n3, G.n4, views, capacity=R0.capacity)
    target = torch.rand_like(R.rgb)
    R.step(G, target)
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in R.grads.items()}
    img = R.rgb.clone()
    gs = raster.GraphedStep(R, G, target)
    for k in R.grads:
        R.grads[k].zero_()
    R.rgb.zero_()
    gs.replay()
    torch.cuda.synchronize()
    R.check()
    assert torch.equal(img, R.rgb)
    for k in R.grads:
        assert rel_l2(R.grads[k].cpu().numpy(), eager[k].cpu().numpy()) < 1e-5, k


def test_autograd_function(small):
    scene, views, G, R, P, ref = small
    params = [G.t[k] for k in F3 + F4]
    for p in params:
        p.requires_grad_(True)
    try:
        out = raster.HybridRasterize.apply(R, G, *params)
        w = torch.randn_like(out)
        (out * w).sum().backward()
        R.backward(G, w)
        torch.cuda.synchronize()
        for k, p in zip(F3 + F4, params):
            n = G.n3 if k in F3 else G.n4
            # two backward runs differ only by the order of float atomics
            assert rel_l2(p.grad[:n].float().cpu().numpy(), R.grads[k].cpu().numpy()) < 1e-5, k
    finally:
        for p in params:
            p.requires_grad_(False)
            p.grad = None


def test_nonfinite_parameters_are_reported_and_culled(small):
    """A NaN in a Gaussian's geometry or colour coefficients sets status NONFINITE with
    its row and culls that Gaussian (fault injected on the host); the next call on
    clean parameters renders exactly as before."""
    scene, views, G0, R0, P, ref = small
    G = raster.Gaussians.from_scene(scene, "cuda")
    R = raster.Rasterizer(G.n3, G.n4, views, capacity=R0.capacity)
    i = int(np.argmax(P["visible"][G.n4:] == 1))  # a visible 3D Gaussian
    for field, idx, clean in (("log_scale3", (i, 0), float(scene.log_scale3[i, 0])),
                              ("sh3", (i, 0, 1), float(scene.sh3[i, 0, 1]))):
        G.t[field][idx] = float("nan")
        R.forward(G)
        torch.cuda.synchronize()
        code, stage, aux = R.read_status()
        assert code == abi.SPLAT_ERR_NONFINITE, field
        assert abi.STAGES[stage] == "slice_project" and aux == G.n4 + i, field
        assert R.n_tiles[G.n4 + i].item() == 0, field  # culled
        assert torch.isfinite(R.rgb).all(), field
        G.t[field][idx] = clean
    R.forward(G)
    torch.cuda.synchronize()
    R.check()
    assert torch.equal(R.rgb, R0.rgb)


# ---------------------------------------------------------------------------
# Edge cases of the compositing decisions and of the batch
# ---------------------------------------------------------------------------

def test_clamped_opacity_matches_oracle():
    """Gaussians whose alpha_max reaches the 0.99 clamp (opacity logits 4.6-8):
    the forward's clamp and the backward's zero derivative where clamped, against
    the oracle (the random scenes almost never reach the clamp)."""
    scene, views = scenes.small_scene(seed=3, n3=1500, n4=500)
    rng = np.random.default_rng(3)
    for k in ("opacity3", "opacity4"):
        o = getattr(scene, k)
        hi = rng.random(o.shape[0]) < 0.4
        o[hi] = rng.uniform(4.6, 8.0, int(hi.sum())).astype(np.float32)
    G, R = make(scene, views)
    P = O.project(scene, views[0])
    vis = P["visible"] == 1
    assert int((P["alpha"][vis] >= 0.99).sum()) > 100
    ref = O.render(scene, views[0])
    check_image(R, P, ref, views[0])
    dls = loss_grad(R, [ref], [P], views, seed=4)
    check_grads(R, G, scene, [P], views, dls)


def test_power_zero_at_pixel_centres():
    """Means that project exactly onto pixel centres (z = 4, f = 64, x = k / 16):
    there the power is exactly 0, which passes the skip test (power > 0 skips)
    and blends with alpha = alpha_max.  4D Gaussians sliced at their own mu_t
    keep their mean exactly."""
    rng = np.random.default_rng(12)
    view = scenes.identity_view(64, 64, 64.0, 0.5)

    def centred(n):
        k = rng.integers(-28, 29, size=(n, 2))
        return np.concatenate([k / 16.0, np.full((n, 1), 4.0)], axis=1)

    n3, n4 = 120, 60
    scene = scenes.random_scene(rng, n3, n4, centred(n3), centred(n4))
    scene.mean4[:, 3] = 0.5
    P = O.project(scene, view)
    vis = P["visible"] == 1
    assert np.all(P["px"][vis] == np.round(P["px"][vis])) and np.all(P["py"][vis] == np.round(P["py"][vis]))
    G, R = make(scene, [view])
    ref = O.render(scene, view)
    check_image(R, P, ref, view)
    # the centre pixels themselves take part in the comparison
    frag = fragile_pixels(P, ref, view)
    centres = (P["py"][vis].astype(int) * view.W + P["px"][vis].astype(int))
    assert (~frag[centres]).mean() > 0.9
    dls = loss_grad(R, [ref], [P], [view], seed=5)
    check_grads(R, G, scene, [P], [view], dls)


def test_max_batch_sixteen_views_mixed_sizes():
    """The largest batch (16 views) in one launch per stage, sizes from 1x1 to
    67x45 (ragged tiles), distinct cameras and timestamps, with a few Gaussians
    larger than the image; every view against the oracle, gradients summed."""
    rng = np.random.default_rng(21)
    scene, _ = scenes.small_scene(seed=21, n3=600, n4=300)
    for i in range(3):  # large splats covering every tile
        scene.log_scale3[i] = np.float32(-0.3)
        scene.mean3[i] = np.array([0.1 * i, -0.1 * i, 3.0], np.float32)
    sizes = [(1, 1), (16, 16), (17, 9), (33, 31), (64, 48), (15, 17), (67, 45), (40, 40),
             (31, 33), (2, 50), (50, 2), (48, 64), (23, 29), (32, 16), (9, 17), (45, 67)]
    views = []
    for W, H in sizes:
        eye = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.0])
        views.append(scenes.look_at_view(eye, np.array([0.0, 0.0, 4.0]), W, H, 0.9 * max(W, H),
                                         float(rng.uniform(0, 1))))
    assert len(views) == abi.SPLAT_MAX_VIEWS
    G, R = make(scene, views)
    Ps = [O.project(scene, v) for v in views]
    refs = [O.render(scene, v) for v in views]
    for v in range(len(views)):
        check_image(R, Ps[v], refs[v], views[v], v)
    dls = loss_grad(R, refs, Ps, views, seed=6)
    check_grads(R, G, scene, Ps, views, dls)


def test_tile_order_longest_first_changes_nothing(small):
    """splat_bin_sort writes the tiles longest list first (classes of eight per
    power of two: the exponent and the next three bits of the length); the
    compositing kernels take them in that order.  The order is a permutation of
    the tiles, non-increasing by class, and rendering with it or
    in raster order (NULL) gives the same images, T and ends of walks (gradients
    up to the order of their float atomics)."""
    scene, views = scenes.arc_scene(seed=5, n=20000, frac4=0.3, n_views=3, full=(256, 192, 280.0),
                                    half=(120, 96, 130.0))
    G, R = make(scene, views)
    target = torch.rand(R.rgb.shape, generator=torch.Generator(device="cuda").manual_seed(13), device="cuda")
    out = []
    try:
        for use in (True, False):
            if not use:
                R.cbins.tile_order = None
            R.step(G, target)
            torch.cuda.synchronize()
            R.check()
            out.append((R.rgb.clone(), R.final_T.clone(), R.last.clone(), {k: v.clone() for k, v in R.grads.items()}))
            if use:
                order = R.tile_order.cpu().numpy().astype(np.int64)
                rg = R.ranges.cpu().numpy().astype(np.int64).reshape(-1, 2)
    finally:
        R.cbins.tile_order = R.tile_order.data_ptr()
    T = R.total_tiles
    assert np.array_equal(np.sort(order[:T]), np.arange(T))
    length = rg[order[:T], 1] - rg[order[:T], 0]
    e = np.floor(np.log2(np.maximum(length, 1))).astype(np.int64)
    frac = np.floor((np.maximum(length, 1) / 2.0 ** e - 1.0) * 8).astype(np.int64)
    cls = np.where(length > 0, 1 + 8 * e + frac, 0)
    assert np.all(np.diff(cls) <= 0) and cls[0] > cls[-1]
    # each class spans less than a factor 9/8 of lengths
    for c in np.unique(cls[cls > 0]):
        sel = length[cls == c]
        assert sel.max() < sel.min() * 9 / 8 + 1
    (rgb0, T0, l0, g0), (rgb1, T1, l1, g1) = out
    assert torch.equal(rgb0, rgb1) and torch.equal(T0, T1) and torch.equal(l0, l1)
    for k in g0:
        assert rel_l2(g1[k].cpu().numpy(), g0[k].cpu().numpy()) < 1e-6, k
