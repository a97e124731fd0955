"""FP64 CPU oracle for the hybrid 3D-4D Gaussian rasterizer (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg may import this package.  It shares no code with the CUDA path;
its inputs are the seeded float32 scenes, widened to float64 exactly.

Functions follow the paper's equations (see oracle.c for the citations):
  rot4 (Eq. 4), cov3 (Eq. 2), cov4, slice (Eq. 5/6 + temporal factor),
  sh_basis (real SH, degree 3), project (cull + EWA + SH, Alg. 1),
  render (Eq. 3 as the plain per-pixel definition), render_bwd (reverse mode),
  matrix_to_quat (Eq. 9), convert (Sec. 4.1-4.2), stable_sort_u64; in numpy:
  adam_step (the optimizer of the training step, Kingma and Ba 2015),
  densify_stats and densify_set (the 3DGS densification rules, Sec. 4.3).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


class _G3(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean", _dp), ("log_scale", _dp), ("quat", _dp),
                ("opacity", _dp), ("sh", _dp)]


class _G4(C.Structure):
    _fields_ = [("n", C.c_int64), ("mean", _dp), ("log_scale", _dp), ("ql", _dp), ("qr", _dp),
                ("opacity", _dp), ("sh", _dp), ("n_time", C.c_int64)]


class _View(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("T", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("W", C.c_int32), ("H", C.c_int32),
                ("pad0", C.c_int32), ("pad1", C.c_int32), ("time", C.c_double), ("z_near", C.c_double),
                ("bg", C.c_double * 3)]


PROJ_DTYPE = np.dtype([
    ("px", "f8"), ("py", "f8"), ("depth", "f8"), ("conic", "f8", 3), ("alpha", "f8"), ("rgb", "f8", 3),
    ("margin_fwd", "f8"), ("margin_grad", "f8"),
    ("radius", "i4"), ("rect", "i4", 4), ("visible", "i4"), ("n_tiles", "i4"), ("pad", "i4"),
    ("r3", "f8"), ("margin_cull", "f8"),
], align=True)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_rot4.argtypes = [_dp, _dp, _dp]
        L.oracle_cov3.argtypes = [_dp, _dp, _dp]
        L.oracle_cov4.argtypes = [_dp, _dp, _dp, _dp]
        L.oracle_quat_to_R3.argtypes = [_dp, _dp]
        L.oracle_slice.argtypes = [_dp, _dp, C.c_double, _dp, _dp, _dp]
        L.oracle_sh_basis.argtypes = [_dp, _dp, _dp]
        L.oracle_project.argtypes = [C.POINTER(_G3), C.POINTER(_G4), C.POINTER(_View), C.c_void_p]
        L.oracle_render.argtypes = [C.POINTER(_G3), C.POINTER(_G4), C.POINTER(_View), _i64p, C.c_int64,
                                    _dp, _dp, _i32p, _dp]
        L.oracle_render_bwd.argtypes = [C.POINTER(_G3), C.POINTER(_G4), C.POINTER(_View), _dp] + [_dp] * 12
        L.oracle_tile_list.argtypes = [C.POINTER(_G3), C.POINTER(_G4), C.POINTER(_View), C.c_int, C.c_int, _i64p]
        L.oracle_tile_list.restype = C.c_int64
        L.oracle_matrix_to_quat.argtypes = [_dp, _dp]
        L.oracle_convert.argtypes = [C.POINTER(_G4), C.c_double, _i32p, _dp, _dp, _dp, _dp, _dp, _i64p]
        L.oracle_convert.restype = C.c_int64
        L.oracle_stable_sort_u64.argtypes = [C.POINTER(C.c_uint64), C.c_int64, _i64p]
        L.oracle_num_threads.restype = C.c_int
        L.oracle_set_num_threads.argtypes = [C.c_int]
        L.oracle_set_margin_impact.argtypes = [C.c_double]
        _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return a.ctypes.data_as(_dp)


def _get(scene, name):
    return scene[name] if isinstance(scene, dict) else getattr(scene, name)


class _Packed:
    """Keeps float64 copies alive while C holds pointers into them."""

    def __init__(self, scene):
        self.m3 = _f64(_get(scene, "mean3"), (-1, 3))
        self.l3 = _f64(_get(scene, "log_scale3"), (-1, 3))
        self.q3 = _f64(_get(scene, "quat3"), (-1, 4))
        self.o3 = _f64(_get(scene, "opacity3"), (-1,))
        self.s3 = _f64(_get(scene, "sh3"), (-1, 16, 3))
        self.m4 = _f64(_get(scene, "mean4"), (-1, 4))
        self.l4 = _f64(_get(scene, "log_scale4"), (-1, 4))
        self.ql = _f64(_get(scene, "ql"), (-1, 4))
        self.qr = _f64(_get(scene, "qr"), (-1, 4))
        self.o4 = _f64(_get(scene, "opacity4"), (-1,))
        # sh4: [n][16 (T + 1)][3], the coefficient blocks of the T + 1 time frequencies
        self.s4 = _f64(_get(scene, "sh4"))
        self.n_time = self.s4.shape[1] // 16 - 1 if self.s4.ndim == 3 and self.s4.shape[0] else 0
        self.s4 = self.s4.reshape(-1, 16 * (self.n_time + 1), 3)
        self.n3 = self.m3.shape[0]
        self.n4 = self.m4.shape[0]
        self.g3 = _G3(self.n3, _p(self.m3), _p(self.l3), _p(self.q3), _p(self.o3), _p(self.s3))
        self.g4 = _G4(self.n4, _p(self.m4), _p(self.l4), _p(self.ql), _p(self.qr), _p(self.o4), _p(self.s4),
                      self.n_time)


def _view(v) -> _View:
    out = _View()
    R = np.asarray(v.R, dtype=np.float64).reshape(9)
    T = np.asarray(v.T, dtype=np.float64).reshape(3)
    for k in range(9):
        out.R[k] = float(R[k])
    for k in range(3):
        out.T[k] = float(T[k])
        out.bg[k] = float(v.bg[k])
    out.fx, out.fy, out.cx, out.cy = float(v.fx), float(v.fy), float(v.cx), float(v.cy)
    out.W, out.H = int(v.W), int(v.H)
    out.time = float(v.t)
    out.z_near = float(v.z_near)
    return out


# ---------------------------------------------------------------------------
# Equations
# ---------------------------------------------------------------------------

def quat_to_R3(q):
    q = _f64(q, (4,))
    R = np.zeros(9)
    lib().oracle_quat_to_R3(_p(q), _p(R))
    return R.reshape(3, 3)


def rot4(ql, qr):
    """Eq. 4 with both quaternions normalised."""
    ql, qr = _f64(ql, (4,)), _f64(qr, (4,))
    R = np.zeros(16)
    lib().oracle_rot4(_p(ql), _p(qr), _p(R))
    return R.reshape(4, 4)


def cov3(quat, log_scale):
    """Eq. 2."""
    q, s = _f64(quat, (4,)), _f64(log_scale, (3,))
    S = np.zeros(9)
    lib().oracle_cov3(_p(q), _p(s), _p(S))
    return S.reshape(3, 3)


def cov4(ql, qr, log_scale):
    a, b, s = _f64(ql, (4,)), _f64(qr, (4,)), _f64(log_scale, (4,))
    S = np.zeros(16)
    lib().oracle_cov4(_p(a), _p(b), _p(s), _p(S))
    return S.reshape(4, 4)


def slice(mean4, Sigma4, t):
    """Eq. 5/6 and the temporal factor: returns (mu3, cov3, p_t)."""
    m, S = _f64(mean4, (4,)), _f64(Sigma4, (16,))
    mu, cv, p = np.zeros(3), np.zeros(9), np.zeros(1)
    lib().oracle_slice(_p(m), _p(S), float(t), _p(mu), _p(cv), _p(p))
    return mu, cv.reshape(3, 3), float(p[0])


def sh_basis(d, with_grad=False):
    d = _f64(d, (3,))
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib().oracle_sh_basis(_p(d), _p(Y), _p(dY) if with_grad else None)
    return (Y, dY.reshape(16, 3)) if with_grad else Y


def matrix_to_quat(R):
    """Eq. 9 (with the largest-diagonal fallback), normalised, w >= 0."""
    R = _f64(R, (9,))
    q = np.zeros(4)
    lib().oracle_matrix_to_quat(_p(R), _p(q))
    return q


# ---------------------------------------------------------------------------
# Rendering
# ---------------------------------------------------------------------------

def project(scene, view):
    """Per merged Gaussian (4D first, then 3D): a PROJ_DTYPE record."""
    pk = _Packed(scene)
    out = np.zeros(pk.n3 + pk.n4, dtype=PROJ_DTYPE)
    v = _view(view)
    lib().oracle_project(C.byref(pk.g3), C.byref(pk.g4), C.byref(v), out.ctypes.data_as(C.c_void_p))
    return out


def render(scene, view, pixels=None):
    """Eq. 3 as the plain definition.  pixels: flat indices y*W+x (None = all).
    Returns dict rgb [3, npix], T [npix], last [npix] (where the walk ends: the
    list index of the entry that would take T below 1e-4, else the list
    length), the per-decision margins
    (dict 'margins': power, alpha, stop, tie, clamp, tie3), margin_fwd (min of
    the first four) and margin_grad (the clamp).  'tie' is the relative depth gap
    of two touching Gaussians of which one is 4D; 'tie3' the distance of a 3D
    pair's depth to an FP32 rounding boundary when their FP32 keys are at most
    one step apart."""
    pk = _Packed(scene)
    v = _view(view)
    if pixels is None:
        npix = int(view.W) * int(view.H)
        pix_p = None
    else:
        pixels = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        npix = pixels.shape[0]
        pix_p = pixels.ctypes.data_as(_i64p)
    rgb = np.zeros((3, npix))
    T = np.zeros(npix)
    last = np.zeros(npix, dtype=np.int32)
    mg = np.zeros((6, npix))
    lib().oracle_render(C.byref(pk.g3), C.byref(pk.g4), C.byref(v), pix_p, npix, _p(rgb), _p(T),
                        last.ctypes.data_as(_i32p), _p(mg))
    names = ("power", "alpha", "stop", "tie", "clamp", "tie3")
    return {"rgb": rgb, "T": T, "last": last, "margins": dict(zip(names, mg)),
            "margin_fwd": mg[:4].min(0), "margin_grad": mg[4]}


def tile_list(scene, view, tx, ty):
    pk = _Packed(scene)
    v = _view(view)
    ids = np.zeros(max(1, pk.n3 + pk.n4), dtype=np.int64)
    m = lib().oracle_tile_list(C.byref(pk.g3), C.byref(pk.g4), C.byref(v), int(tx), int(ty),
                               ids.ctypes.data_as(_i64p))
    return ids[:m]


def render_bwd(scene, view, dLdC):
    """Reverse mode for one view.  dLdC: [3, H, W].  Returns a dict of float64
    gradients shaped like the scene arrays, plus 'dproj' [n, 9]."""
    pk = _Packed(scene)
    v = _view(view)
    g = _f64(dLdC, (3 * int(view.W) * int(view.H),))
    out = {
        "mean3": np.zeros((pk.n3, 3)), "log_scale3": np.zeros((pk.n3, 3)), "quat3": np.zeros((pk.n3, 4)),
        "opacity3": np.zeros(pk.n3), "sh3": np.zeros((pk.n3, 16, 3)),
        "mean4": np.zeros((pk.n4, 4)), "log_scale4": np.zeros((pk.n4, 4)), "ql": np.zeros((pk.n4, 4)),
        "qr": np.zeros((pk.n4, 4)), "opacity4": np.zeros(pk.n4), "sh4": np.zeros((pk.n4, 16 * (pk.n_time + 1), 3)),
        "dproj": np.zeros((pk.n3 + pk.n4, 9)),
    }
    lib().oracle_render_bwd(C.byref(pk.g3), C.byref(pk.g4), C.byref(v), _p(g),
                            _p(out["mean3"]), _p(out["log_scale3"]), _p(out["quat3"]), _p(out["opacity3"]),
                            _p(out["sh3"]), _p(out["mean4"]), _p(out["log_scale4"]), _p(out["ql"]),
                            _p(out["qr"]), _p(out["opacity4"]), _p(out["sh4"]), _p(out["dproj"]))
    return out


def adam_step(p, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One step of Adam (Kingma and Ba, 2015, Algorithm 1) in FP64 -- the
    optimizer of the 3DGS / 4DGS training that the paper's training builds on
    (Sec. 4.3): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, bias-corrected
    m / (1 - b1^t) and v / (1 - b2^t), p -= lr m_hat / (sqrt(v_hat) + eps).
    lr may be an array broadcast against p.  Returns (p, m, v)."""
    p, m, v, g = (np.asarray(x, dtype=np.float64) for x in (p, m, v, g))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - np.asarray(lr, dtype=np.float64) * mh / (np.sqrt(vh) + eps), m, v


FIELDS3 = ("mean3", "log_scale3", "quat3", "opacity3", "sh3")
FIELDS4 = ("mean4", "log_scale4", "ql", "qr", "opacity4", "sh4")


def densify_stats(dproj_xy, visible, W, H):
    """Densification statistics of one view: per Gaussian |dL/d(NDC mean)| =
    |(dL/dpx W/2, dL/dpy H/2)| where the view sees it, and the count (0/1)."""
    g = np.asarray(dproj_xy, dtype=np.float64) * np.array([0.5 * W, 0.5 * H])
    vis = np.asarray(visible, dtype=bool)
    return np.where(vis, np.sqrt((g * g).sum(1)), 0.0), vis.astype(np.float64)


def densify_set(params, m, v, accum, count, noise, grad_threshold, dense_scale, min_opacity, split_shrink,
                four_d):
    """The 3DGS densification rules the paper adopts (Sec. 4.3), on one set, FP64.
    params / m / v: dicts of the set's fields (FIELDS3 or FIELDS4), n rows.
    sigmoid(o) < min_opacity: removed.  Otherwise mean statistic accum / count
    >= grad_threshold: cloned when max(exp(s_x, s_y, s_z)) <= dense_scale, else
    split into two Gaussians at mean + M z_h (M = R diag(exp(s)), R the
    rotation of the quaternion (3D) or of Eq. 4 (4D), z_h = noise[i, h]) with
    every log-scale lowered by split_shrink.  Returns (params, m, v) of the new
    set: kept rows, clones, children; new rows with zero moments."""
    fields = FIELDS4 if four_d else FIELDS3
    P = {k: np.asarray(params[k], dtype=np.float64) for k in fields}
    n = P[fields[0]].shape[0]
    o = P["opacity4" if four_d else "opacity3"]
    ls = P["log_scale4" if four_d else "log_scale3"]
    mu = P["mean4" if four_d else "mean3"]
    op = 1.0 / (1.0 + np.exp(-o))
    c = np.asarray(count, dtype=np.float64)
    avg = np.where(c > 0, np.asarray(accum, dtype=np.float64) / np.where(c > 0, c, 1.0), 0.0)
    alive = op >= min_opacity
    dens = alive & (avg >= grad_threshold)
    small = np.exp(ls[:, :3].max(1)) <= dense_scale
    clone, split = dens & small, dens & ~small
    keep = alive & ~split
    kids = {k: [] for k in fields}
    for i in np.nonzero(split)[0]:
        if four_d:
            R = rot4(P["ql"][i], P["qr"][i])
        else:
            q = P["quat3"][i]
            R = quat_to_R3(q / np.linalg.norm(q))
        M = R * np.exp(ls[i])[None, :]
        for h in range(2):
            for k in fields:
                kids[k].append(P[k][i].copy())
            kids["mean4" if four_d else "mean3"][-1] = mu[i] + M @ np.asarray(noise[i, h], dtype=np.float64)
            kids["log_scale4" if four_d else "log_scale3"][-1] = ls[i] - split_shrink
    out_p, out_m, out_v = {}, {}, {}
    for k in fields:
        shape = P[k].shape[1:]
        kid = np.array(kids[k]).reshape((-1,) + shape)
        out_p[k] = np.concatenate([P[k][keep], P[k][clone], kid], 0)
        zeros = np.zeros((int(clone.sum()) + kid.shape[0],) + shape)
        out_m[k] = np.concatenate([np.asarray(m[k], dtype=np.float64)[keep], zeros], 0)
        out_v[k] = np.concatenate([np.asarray(v[k], dtype=np.float64)[keep], zeros], 0)
    return out_p, out_m, out_v


def convert(scene, tau):
    """Sec. 4.1-4.2 on the 4D set: returns (moved mask, appended 3D arrays, kept 4D indices)."""
    pk = _Packed(scene)
    n4 = pk.n4
    moved = np.zeros(n4, dtype=np.int32)
    m3, l3, q3 = np.zeros((n4, 3)), np.zeros((n4, 3)), np.zeros((n4, 4))
    o3, s3 = np.zeros(n4), np.zeros((n4, 16, 3))
    keep = np.zeros(max(1, n4), dtype=np.int64)
    nm = lib().oracle_convert(C.byref(pk.g4), float(tau), moved.ctypes.data_as(_i32p), _p(m3), _p(l3), _p(q3),
                              _p(o3), _p(s3), keep.ctypes.data_as(_i64p))
    app = {"mean3": m3[:nm], "log_scale3": l3[:nm], "quat3": q3[:nm], "opacity3": o3[:nm], "sh3": s3[:nm]}
    return moved.astype(bool), app, keep[: n4 - nm]


def stable_sort_u64(keys):
    k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
    perm = np.zeros(k.shape[0], dtype=np.int64)
    lib().oracle_stable_sort_u64(k.ctypes.data_as(C.POINTER(C.c_uint64)), k.shape[0], perm.ctypes.data_as(_i64p))
    return perm


def set_margin_impact(impact: float) -> None:
    """Record a forward decision's margin only when flipping it could change the
    pixel by at least `impact` (0 = every decision)."""
    lib().oracle_set_margin_impact(float(impact))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def tile_keys(proj, view, depth_f32=None):
    """The (tile << 32 | float32 depth bits) keys that DuplicateWithKeys emits for one
    view, in emission order (merged index, then tiles row major), with the merged
    index of each.  depth_f32 overrides the depth (float32 array) used for the key."""
    TX = (int(view.W) + 15) // 16
    keys, ids = [], []
    dep = np.asarray(proj["depth"], dtype=np.float32) if depth_f32 is None else np.asarray(depth_f32, np.float32)
    dbits = dep.view(np.uint32).astype(np.uint64)
    for i in np.nonzero(proj["visible"])[0]:
        x0, y0, x1, y1 = proj["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                keys.append((np.uint64(ty * TX + tx) << np.uint64(32)) | dbits[i])
                ids.append(i)
    return np.asarray(keys, dtype=np.uint64), np.asarray(ids, dtype=np.int64)
