"""Seeded synthetic scenes and cameras shaped like the paper's workloads.

This module only draws random numbers and builds pinhole cameras; it holds
none of the rasterizer's arithmetic.  Both the CUDA path and the FP64 CPU
oracle take their inputs from here, so they see bit-identical parameters
(float32 arrays; the oracle widens them to float64 exactly).

Parameter distributions (all raw, before activation):
  log-scales ~ N(-3, 0.5); 4D time log-scale ~ N(-2, 0.5); mu_t ~ U[0, 1]
  quaternions: normalised N(0, I_4) (3D q, 4D q_l and q_r)
  opacity logit ~ N(0, 1)
  SH degree 3: DC ~ N(0, 1), the 15 higher coefficients ~ N(0, 0.1)

The paper's datasets (N3V multi-view video at 2704x2028 downsampled to
1352x1014, ~300k initial COLMAP points, 300-frame sequences) are not
available; these scenes stand in for them with the same image sizes,
Gaussian counts and frame grids.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SH_COEFFS = 16  # degree 3


@dataclasses.dataclass
class Scene:
    """A mixed set of static (3D) and dynamic (4D) Gaussians, float32, host memory."""
    mean3: np.ndarray       # [n3, 3]
    log_scale3: np.ndarray  # [n3, 3]
    quat3: np.ndarray       # [n3, 4]  (w, x, y, z)
    opacity3: np.ndarray    # [n3]     logit
    sh3: np.ndarray         # [n3, 16, 3]
    mean4: np.ndarray       # [n4, 4]  (x, y, z, t)
    log_scale4: np.ndarray  # [n4, 4]
    ql: np.ndarray          # [n4, 4]  (a, b, c, d)
    qr: np.ndarray          # [n4, 4]  (p, q, r, s)
    opacity4: np.ndarray    # [n4]
    sh4: np.ndarray         # [n4, 16, 3]

    @property
    def n3(self) -> int:
        return int(self.mean3.shape[0])

    @property
    def n4(self) -> int:
        return int(self.mean4.shape[0])

    @property
    def n(self) -> int:
        return self.n3 + self.n4

    def arrays(self):
        return {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}

    def astype(self, dtype) -> "Scene":
        return Scene(**{k: np.ascontiguousarray(v, dtype=dtype) for k, v in self.arrays().items()})


@dataclasses.dataclass
class View:
    """Pinhole camera: x_cam = R x_world + T, u = fx x/z + cx, v = fy y/z + cy."""
    R: np.ndarray           # [3, 3] world -> camera rotation
    T: np.ndarray           # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    t: float                # timestamp the 4D Gaussians are sliced at
    z_near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng: np.random.Generator, n: int) -> np.ndarray:
    sh = rng.normal(0.0, 0.1, size=(n, SH_COEFFS, 3))
    sh[:, 0, :] = rng.standard_normal((n, 3))
    return sh


def random_scene(rng: np.random.Generator, n3: int, n4: int, means3: np.ndarray, means4_xyz: np.ndarray) -> Scene:
    """Gaussians at the given positions with the common parameter distributions."""
    mean4 = np.concatenate([means4_xyz, rng.uniform(0.0, 1.0, size=(n4, 1))], axis=1)
    log4 = rng.normal(-3.0, 0.5, size=(n4, 4))
    log4[:, 3] = rng.normal(-2.0, 0.5, size=n4)
    s = Scene(
        mean3=means3,
        log_scale3=rng.normal(-3.0, 0.5, size=(n3, 3)),
        quat3=_unit_quats(rng, n3),
        opacity3=rng.standard_normal(n3),
        sh3=_sh(rng, n3),
        mean4=mean4,
        log_scale4=log4,
        ql=_unit_quats(rng, n4),
        qr=_unit_quats(rng, n4),
        opacity4=rng.standard_normal(n4),
        sh4=_sh(rng, n4),
    )
    return s.astype(np.float32)


def frustum_means(rng: np.random.Generator, n: int, z_lo: float, z_hi: float, half_w: float, half_h: float) -> np.ndarray:
    """Uniform depth in [z_lo, z_hi]; x, y uniform over the frustum cross-section at that depth
    (half_w, half_h are the half extents at z = 1)."""
    z = rng.uniform(z_lo, z_hi, size=n)
    x = rng.uniform(-1.0, 1.0, size=n) * half_w * z
    y = rng.uniform(-1.0, 1.0, size=n) * half_h * z
    return np.stack([x, y, z], axis=1)


def identity_view(W: int, H: int, f: float, t: float) -> View:
    return View(R=np.eye(3, dtype=np.float32), T=np.zeros(3, dtype=np.float32), fx=f, fy=f,
                cx=W / 2.0, cy=H / 2.0, W=W, H=H, t=t)


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------

def small_scene(seed: int = 0, n3: int = 3072, n4: int = 1024):
    """One 128x128 view (8x8 tiles), fx = fy = 128, camera at the origin looking
    down +z, t = 0.5; means uniform in [-1, 1]^2 x [2, 6]."""
    rng = np.random.default_rng(seed)
    def means(n):
        return np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 6, n)], axis=1)
    m3 = means(n3)
    m4 = means(n4)
    scene = random_scene(rng, n3, n4, m3, m4)
    view = identity_view(128, 128, 128.0, 0.5)
    return scene, [view]


def frames(n_frames: int = 300) -> np.ndarray:
    return np.arange(n_frames, dtype=np.float64) / (n_frames - 1)


def video_scene(seed: int = 1, n3: int = 200_000, n4: int = 100_000, W: int = 1352, H: int = 1014,
                f: float = 1460.0):
    """One 1352x1014 view, fx = fy = 1460, depth U[1, 20], x/y uniform over the
    frustum cross-section; t drawn from a 300-frame grid."""
    rng = np.random.default_rng(seed)
    hw, hh = W / (2 * f), H / (2 * f)
    m3 = frustum_means(rng, n3, 1.0, 20.0, hw, hh)
    m4 = frustum_means(rng, n4, 1.0, 20.0, hw, hh)
    scene = random_scene(rng, n3, n4, m3, m4)
    t = float(frames()[rng.integers(0, 300)])
    view = identity_view(W, H, f, t)
    return scene, [view]


def jittered_views(base: View, n_views: int, seed: int, max_angle_deg: float = 3.0,
                   max_shift: float = 0.3) -> List[View]:
    """n_views cameras near `base`: small random rotations and translations,
    distinct timestamps from the 300-frame grid."""
    rng = np.random.default_rng(seed)
    grid = frames()
    out = []
    for v in range(n_views):
        if v == 0:
            R = np.asarray(base.R, dtype=np.float64)
            T = np.asarray(base.T, dtype=np.float64)
        else:
            axis = rng.standard_normal(3)
            axis /= np.linalg.norm(axis)
            ang = math.radians(rng.uniform(-max_angle_deg, max_angle_deg))
            K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
            dR = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
            R = dR @ np.asarray(base.R, dtype=np.float64)
            T = np.asarray(base.T, dtype=np.float64) + rng.uniform(-max_shift, max_shift, 3)
        t = float(grid[rng.integers(0, len(grid))])
        out.append(dataclasses.replace(base, R=R.astype(np.float32), T=T.astype(np.float32), t=t))
    return out


def look_at_view(eye: np.ndarray, target: np.ndarray, W: int, H: int, f: float, t: float) -> View:
    """Camera at `eye` looking at `target` (+z forward, y down)."""
    fwd = target - eye
    fwd = fwd / np.linalg.norm(fwd)
    up = np.array([0.0, -1.0, 0.0])
    right = np.cross(up, fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=0)
    T = -R @ eye
    return View(R=R.astype(np.float32), T=T.astype(np.float32), fx=f, fy=f, cx=W / 2.0, cy=H / 2.0,
                W=W, H=H, t=t)


def arc_scene(seed: int = 2, n: int = 500_000, frac4: float = 0.3, n_views: int = 8,
              full=(1352, 1014, 1460.0), half=(676, 507, 730.0)):
    """World means U[-5, 5]^3; cameras on a 120-degree arc of radius 11 about the
    origin, looking at it; even views full resolution, odd views half; distinct
    timestamps t_v = (v + U[0,1)) / n_views."""
    rng = np.random.default_rng(seed)
    n4 = int(round(n * frac4))
    n3 = n - n4
    m3 = rng.uniform(-5, 5, size=(n3, 3))
    m4 = rng.uniform(-5, 5, size=(n4, 3))
    scene = random_scene(rng, n3, n4, m3, m4)
    views = []
    for v in range(n_views):
        ang = math.radians(-60.0 + 120.0 * v / max(1, n_views - 1))
        eye = np.array([11.0 * math.sin(ang), 0.0, -11.0 * math.cos(ang)])
        W, H, f = full if v % 2 == 0 else half
        t = (v + rng.uniform(0.0, 1.0)) / n_views
        views.append(look_at_view(eye, np.zeros(3), W, H, f, t))
    return scene, views


def training_scene(seed: int = 4, n: int = 300_000, frac_static: float = 0.7) -> Scene:
    """Every Gaussian 4D (the paper starts from a full 4D model, Sec. 4.3), world
    means U[-5, 5]^3.  A fraction frac_static has the wide time scale of a
    static Gaussian, log s_t ~ N(0.5, 0.3) (exp(s_t) > 1 for 95% of them), the
    rest the narrow one of the common distribution, log s_t ~ N(-2, 0.5): a
    conversion pass with tau = 1 leaves about 1 - frac_static of them 4D, the
    mix the paper's trained models reach."""
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, 0, n, np.zeros((0, 3)), rng.uniform(-5, 5, size=(n, 3)))
    wide = rng.uniform(0.0, 1.0, size=n) < frac_static
    st = scene.log_scale4[:, 3].astype(np.float64)
    st[wide] = rng.normal(0.5, 0.3, size=int(wide.sum()))
    scene.log_scale4[:, 3] = st.astype(np.float32)
    return scene


def random_arc_views(rng: np.random.Generator, n_views: int, W: int = 1352, H: int = 1014, f: float = 1460.0,
                     radius: float = 11.0, n_frames: int = 300) -> List[View]:
    """Training batch: cameras at random angles of a 120-degree arc of the given
    radius about the origin, looking at it, each at a random frame of the
    sequence."""
    grid = frames(n_frames)
    out = []
    for _ in range(n_views):
        ang = math.radians(rng.uniform(-60.0, 60.0))
        eye = np.array([radius * math.sin(ang), rng.uniform(-1.0, 1.0), -radius * math.cos(ang)])
        out.append(look_at_view(eye, np.zeros(3), W, H, f, float(grid[rng.integers(0, n_frames)])))
    return out


def subset(scene: Scene, idx3: Optional[Sequence[int]] = None, idx4: Optional[Sequence[int]] = None) -> Scene:
    a = scene.arrays()
    out = {}
    for k, v in a.items():
        sel = idx4 if k in ("mean4", "log_scale4", "ql", "qr", "opacity4", "sh4") else idx3
        out[k] = np.ascontiguousarray(v if sel is None else v[np.asarray(sel, dtype=np.int64)])
    return Scene(**out)


def empty_scene() -> Scene:
    z = np.zeros
    return Scene(mean3=z((0, 3), np.float32), log_scale3=z((0, 3), np.float32), quat3=z((0, 4), np.float32),
                 opacity3=z((0,), np.float32), sh3=z((0, 16, 3), np.float32),
                 mean4=z((0, 4), np.float32), log_scale4=z((0, 4), np.float32), ql=z((0, 4), np.float32),
                 qr=z((0, 4), np.float32), opacity4=z((0,), np.float32), sh4=z((0, 16, 3), np.float32))
