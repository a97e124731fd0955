"""Helpers of the GPU-vs-oracle parity tests.

An FP32 kernel and the FP64 oracle can legitimately take a discrete decision
(cull, radius ceil, tile-rectangle floor/ceil, alpha skip, transmittance
stop, depth order of two touching Gaussians) differently when the decided
quantity lies within FP32 rounding of its threshold.  The oracle reports the
relative distance of every decision to its threshold; these helpers turn that
into masks of pixels / Gaussians whose result is not unique at FP32 and
count them.  Everything else must match within the stated tolerance.
"""
import json
import math
import os

import numpy as np

import oracle as O

# a flipped decision counts only if it can move a pixel by half the tolerance
O.set_margin_impact(1e-4)

# Relative windows of FP32 rounding per decision type.  Each is a few times
# the error an FP32 evaluation of that quantity carries:
#  - rectangle edges (px +- r)/16: px carries ~1e-7 relative error
#  - radius 3 sqrt(lambda): lambda carries a few 1e-7 relative error
#  - cull: alpha_max = sigmoid(o) p(t), p(t) = exp(-dt^2/2S) carries ~5e-6
#  - per pixel: power (conic ~1e-6 relative, |power| <= 5.5) -> alpha ~1e-5;
#    transmittance accumulates ~1e-7 per blended Gaussian; depth ~2e-7
EPS_RECT = 1e-6
EPS_RADIUS = 1e-6
EPS_CULL = 3e-5
# tie3: a 3D Gaussian's depth is rounded to FP32 exactly by the kernel's
# compensated dot product, up to ~1e-12 of the depth for the scenes here
EPS_PIXEL = {"power": 1e-5, "alpha": 5e-5, "stop": 5e-5, "tie": 1e-6, "tie3": 1e-10}
EPS_CLAMP = 5e-5      # alpha clamp at 0.99: a kink of the gradient only
EPS_GRAD_GAUSS = 3e-5  # Jacobian clamp, rgb clamp: kinks of one Gaussian's gradient
RGB_TOL = 2e-4        # max-abs on colours in [0, 1]
# Bound of the pixels set aside as not unique at FP32 among n compared:
# FRAGILE_FRAC n + FRAGILE_SLACK.  A pixel is set aside when one of the
# decisions along its walk lies within its window (a few times that decision's
# FP32 error) of its threshold, so the expected count grows with the
# decisions per walk: measured 0.04-0.09% of the small scenes' images and up
# to about 1% of the dense full-size samples.  The bounds are about three
# times that, so that an oracle margin that sets aside too much fails.
FRAGILE_FRAC = {"small": 0.003, "dense": 0.01}
FRAGILE_SLACK = 3


def fragile_bound(n, kind="small"):
    return FRAGILE_FRAC[kind] * n + FRAGILE_SLACK
GRAD_RTOL = 1e-3      # relative L2 per gradient tensor


def _int_margin(q):
    q = np.asarray(q, np.float64)
    return np.abs(q - np.rint(q)) / np.maximum(1.0, np.abs(q))


def gaussian_flags(P):
    """Per Gaussian: (any decision fragile, cull fragile, radius fragile)."""
    finite = np.isfinite(P["r3"]) & (P["depth"] > 0)
    cull = P["margin_cull"] < EPS_CULL
    rad = finite & (_int_margin(np.where(finite, P["r3"], 0.5)) < EPS_RADIUS)
    r = np.ceil(np.where(finite, P["r3"], 0.0))
    edges = np.zeros(len(P), bool)
    for q in ((P["px"] - r) / 16, (P["px"] + r) / 16, (P["py"] - r) / 16, (P["py"] + r) / 16):
        edges |= finite & (_int_margin(np.where(finite, q, 0.5)) < EPS_RECT)
    relevant = (P["visible"] == 1) | cull
    return relevant & (cull | rad | edges), cull, rad


def fragile_gaussians(P):
    return gaussian_flags(P)[0]


def _alt_floor(q, eps):
    w = eps * max(1.0, abs(q))
    return {math.floor(q - w), math.floor(q + w)}


def _alt_ceil(q, eps):
    w = eps * max(1.0, abs(q))
    return {math.ceil(q - w), math.ceil(q + w)}


def _alternative_rects(p, cull, TX, TY):
    """Union and intersection of the tile rectangles over the alternative
    radius / edge decisions of one Gaussian."""
    r3 = p["r3"]
    radii = {math.ceil(r3 * (1 - EPS_RADIUS)), math.ceil(r3 * (1 + EPS_RADIUS))}
    xs0, xs1, ys0, ys1 = set(), set(), set(), set()
    for rr in radii:
        xs0 |= _alt_floor((p["px"] - rr) / 16, EPS_RECT)
        xs1 |= _alt_ceil((p["px"] + rr) / 16, EPS_RECT)
        ys0 |= _alt_floor((p["py"] - rr) / 16, EPS_RECT)
        ys1 |= _alt_ceil((p["py"] + rr) / 16, EPS_RECT)
    cl = lambda v, hi: min(max(v, 0), hi)
    union = (cl(min(xs0), TX), cl(min(ys0), TY), cl(max(xs1), TX), cl(max(ys1), TY))
    inter = (cl(max(xs0), TX), cl(max(ys0), TY), cl(min(xs1), TX), cl(min(ys1), TY))
    if cull or inter[2] <= inter[0] or inter[3] <= inter[1]:
        inter = (0, 0, 0, 0)
    return union, inter


def uncertain_tiles(P, view):
    """Boolean [TY, TX]: tiles whose membership in some Gaussian's rectangle
    could flip (union minus intersection over the alternative decisions)."""
    TX, TY = (view.W + 15) // 16, (view.H + 15) // 16
    bad = np.zeros((TY, TX), bool)
    frag, cull, rad = gaussian_flags(P)
    for i in np.nonzero(frag)[0]:
        (ux0, uy0, ux1, uy1), (ix0, iy0, ix1, iy1) = _alternative_rects(P[i], cull[i], TX, TY)
        union = np.zeros((TY, TX), bool)
        union[uy0:uy1, ux0:ux1] = True
        union[iy0:iy1, ix0:ix1] = False
        bad |= union
    return bad


def uncertain_pixels(P, view, pix):
    """Of the flat pixel indices `pix`, those inside a tile whose membership in a
    Gaussian's rectangle could flip AND where that Gaussian reaches alpha >= 1/255
    (only there can the flip change the pixel)."""
    TX, TY = (view.W + 15) // 16, (view.H + 15) // 16
    pix = np.asarray(pix, np.int64)
    u = (pix % view.W).astype(np.float64)
    v = (pix // view.W).astype(np.float64)
    tx, ty = (pix % view.W) // 16, (pix // view.W) // 16
    out = np.zeros(len(pix), bool)
    frag, cull, rad = gaussian_flags(P)
    for i in np.nonzero(frag)[0]:
        p = P[i]
        (ux0, uy0, ux1, uy1), (ix0, iy0, ix1, iy1) = _alternative_rects(p, cull[i], TX, TY)
        inside_u = (tx >= ux0) & (tx < ux1) & (ty >= uy0) & (ty < uy1)
        inside_i = (tx >= ix0) & (tx < ix1) & (ty >= iy0) & (ty < iy1)
        cand = inside_u & ~inside_i
        if not cand.any():
            continue
        dx, dy = p["px"] - u[cand], p["py"] - v[cand]
        a, b, c = p["conic"]
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        alpha = p["alpha"] * np.exp(np.minimum(power, 0.0))
        hit = alpha >= (1.0 / 255.0) * (1 - 1e-3)
        idx = np.nonzero(cand)[0]
        out[idx[hit]] = True
    return out


def pixel_fragile_from_margins(ref):
    m = ref["margins"]
    out = np.zeros_like(m["power"], dtype=bool)
    for k, eps in EPS_PIXEL.items():
        out |= m[k] < eps
    return out


def fragile_pixels(P, ref, view, pix=None):
    """Mask of pixels whose forward result is not unique at FP32 (pix: the flat
    pixel indices ref was rendered at; None = the whole image)."""
    if pix is None:
        pix = np.arange(view.W * view.H)
    return pixel_fragile_from_margins(ref) | uncertain_pixels(P, view, pix)


def grad_fragile_pixels(ref):
    return ref["margins"]["clamp"] < EPS_CLAMP


def grad_fragile_gaussians(P):
    """Gaussians whose own gradient has a kink within its window (Jacobian clamp, rgb clamp)."""
    return P["margin_grad"] < EPS_GRAD_GAUSS


def report(case, **rec):
    """Prints one JSON record of a parity measurement (fragile counts, errors)
    and appends it to the file named by SPLAT_PARITY_REPORT when that is set."""
    line = json.dumps(dict(case=case, **rec))
    print(line)
    path = os.environ.get("SPLAT_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(line + "\n")


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def oracle_grads_views(scene, views, dLdC_per_view):
    """Sum of oracle gradients over views."""
    tot = None
    for v, g in zip(views, dLdC_per_view):
        r = O.render_bwd(scene, v, g)
        r.pop("dproj")
        if tot is None:
            tot = r
        else:
            for k in tot:
                tot[k] = tot[k] + r[k]
    return tot


EPS32 = 2.0 ** -24


def split_mean_tol(mean, log_scale, noise, shrink):
    """Per-element bound of the FP32 error of a densified Gaussian's mean.

    A split child sits at mean + sum_c M_rc z_c with M = R diag(exp(s)) built
    from the normalised quaternion(s) in FP32: each entry of M carries at most
    about 15 roundings relative to exp(s_c) (|R_rc| <= 1), the dot product D
    more and the final add one, so |error_r| <= (16 + D) eps sum_c exp(s_c)
    |z_c| + eps |result_r|.  Bounded here by 32 eps (|result_r| + D max|z|
    max_c exp(s_c)), with the parent's exp(s_c) = exp(child log-scale + shrink).
    Kept and cloned rows are copies (error 0), below any bound."""
    mean = np.asarray(mean, np.float64)
    D = mean.shape[1]
    zmax = float(np.max(np.abs(noise))) if np.size(noise) else 0.0
    smax = np.exp(np.max(np.asarray(log_scale, np.float64), axis=1) + shrink)
    return 32 * EPS32 * (np.abs(mean) + (D * zmax * smax)[:, None])


def assert_split_means(got, want, want_log_scale, noise, shrink, name):
    tol = split_mean_tol(want, want_log_scale, noise, shrink)
    err = np.abs(np.asarray(got, np.float64) - want)
    bad = err > tol
    assert not bad.any(), "%s: %d elements beyond the FP32 bound, worst %s (bound %s)" % (
        name, int(bad.sum()), err[bad].max(), tol[bad][np.argmax(err[bad])])
