"""Helpers of the GPU-vs-oracle parity tests.

An FP32 kernel and the FP64 oracle can legitimately take a discrete decision
(cull, radius ceil, tile-rectangle floor/ceil, alpha skip, transmittance
stop, depth order of two touching Gaussians) differently when the decided
quantity lies within FP32 rounding of its threshold.  The oracle reports the
relative distance of every decision to its threshold; these helpers turn that
into masks of pixels / Gaussians whose result is not unique at FP32 and
count them.  Everything else must match within the stated tolerance.
"""
import math

import numpy as np

import oracle as O

# relative window of FP32 rounding on the decided quantities (conic, power and
# alpha accumulate a few 1e-6 relative error through the projection chain)
EPS_PIXEL = 1e-4
EPS_GAUSS = 2e-5
RGB_TOL = 2e-4        # max-abs on colours in [0, 1]
GRAD_RTOL = 1e-3      # relative L2 per gradient tensor


def _alt_floor(q, eps):
    w = eps * max(1.0, abs(q))
    return {math.floor(q - w), math.floor(q + w)}


def _alt_ceil(q, eps):
    w = eps * max(1.0, abs(q))
    return {math.ceil(q - w), math.ceil(q + w)}


def uncertain_tiles(P, view, eps=EPS_GAUSS):
    """Boolean [TY, TX]: tiles whose membership in some Gaussian's rectangle
    could flip within eps (union minus intersection over the alternatives)."""
    TX, TY = (view.W + 15) // 16, (view.H + 15) // 16
    bad = np.zeros((TY, TX), bool)
    idx = np.nonzero((P["margin_fwd"] < eps) & (P["depth"] > 0))[0]
    for i in idx:
        p = P[i]
        r3 = p["r3"]
        if not np.isfinite(r3) or r3 <= 0:
            continue
        radii = {math.ceil(r3 * (1 - eps)), math.ceil(r3 * (1 + eps))}
        xs0, xs1, ys0, ys1 = set(), set(), set(), set()
        for rr in radii:
            xs0 |= _alt_floor((p["px"] - rr) / 16, eps)
            xs1 |= _alt_ceil((p["px"] + rr) / 16, eps)
            ys0 |= _alt_floor((p["py"] - rr) / 16, eps)
            ys1 |= _alt_ceil((p["py"] + rr) / 16, eps)
        cl = lambda v, hi: min(max(v, 0), hi)
        ux0, ux1 = cl(min(xs0), TX), cl(max(xs1), TX)
        uy0, uy1 = cl(min(ys0), TY), cl(max(ys1), TY)
        ix0, ix1 = cl(max(xs0), TX), cl(min(xs1), TX)
        iy0, iy1 = cl(max(ys0), TY), cl(min(ys1), TY)
        union = np.zeros((TY, TX), bool)
        union[uy0:uy1, ux0:ux1] = True
        inter = np.zeros((TY, TX), bool)
        if p["margin_cull"] >= eps and ix1 > ix0 and iy1 > iy0:
            inter[iy0:iy1, ix0:ix1] = True
        bad |= union & ~inter
    return bad


def fragile_pixels(P, ref, view, eps_pixel=EPS_PIXEL, eps_gauss=EPS_GAUSS):
    """[H*W] mask of pixels whose forward result is not unique at FP32."""
    m = ref["margin_fwd"] < eps_pixel
    tiles = uncertain_tiles(P, view, eps_gauss)
    tile_of_pix = np.kron(tiles, np.ones((16, 16), bool))[: view.H, : view.W].reshape(-1)
    return m | tile_of_pix


def grad_fragile_gaussians(P, eps=EPS_GAUSS):
    """Gaussians whose own gradient has a kink within eps (Jacobian clamp, rgb clamp)."""
    return P["margin_grad"] < eps


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
