"""The oracle's hand-written reverse mode against central finite differences of
its own FP64 forward, on tiny scenes whose discrete decisions all sit well
away from their thresholds (so the forward is smooth under the perturbation)."""
import numpy as np
import pytest

import oracle as O
from paper_2505_13215_gb300 import scenes

FIELDS3 = ["mean3", "log_scale3", "quat3", "opacity3", "sh3"]
FIELDS4 = ["mean4", "log_scale4", "ql", "qr", "opacity4", "sh4"]


def tiny_scene(seed, n3=3, n4=3, W=32, H=32, f=32.0, t=0.5, clamp_case=False):
    rng = np.random.default_rng(seed)
    base, _ = scenes.small_scene(seed=seed, n3=n3, n4=n4)
    sc = {k: v.astype(np.float64).copy() for k, v in base.arrays().items()}
    sc["mean3"][:, :2] = rng.uniform(-0.4, 0.4, (n3, 2))
    sc["mean3"][:, 2] = rng.uniform(2.5, 3.5, n3)
    sc["mean4"][:, :2] = rng.uniform(-0.4, 0.4, (n4, 2))
    sc["mean4"][:, 2] = rng.uniform(2.5, 3.5, n4)
    sc["mean4"][:, 3] = t + rng.uniform(-0.05, 0.05, n4)
    sc["log_scale3"] = rng.normal(-1.8, 0.3, (n3, 3))
    sc["log_scale4"] = rng.normal(-1.8, 0.3, (n4, 4))
    sc["log_scale4"][:, 3] = rng.normal(-1.0, 0.2, n4)
    sc["opacity3"] = rng.normal(0.0, 0.5, n3)
    sc["opacity4"] = rng.normal(0.0, 0.5, n4)
    if clamp_case:
        # a wide Gaussian centred beyond the 1.3 tan(fov/2) clamp that still covers the image
        sc["mean3"][0] = [0.7 * 3.0, 0.1, 3.0]
        sc["log_scale3"][0] = [-1.0, -1.0, -1.0]
    view = scenes.View(R=np.eye(3), T=np.zeros(3), fx=f, fy=f, cx=W / 2 - 0.3, cy=H / 2 + 0.2, W=W, H=H, t=t)
    return sc, view


def loss(sc, view, w):
    return float((O.render(sc, view)["rgb"] * w).sum())


def check_fd(sc, view, rtol=1e-6):
    W, H = view.W, view.H
    r = O.render(sc, view)
    P = O.project(sc, view)
    assert r["margin_fwd"].min() > 1e-4, "scene has a near-threshold decision; choose another seed"
    assert r["margin_grad"].min() > 1e-4
    assert P["margin_fwd"].min() > 1e-4 and P["margin_grad"].min() > 1e-4
    rng = np.random.default_rng(99)
    w = rng.normal(0, 1, (3, W * H))
    g = O.render_bwd(sc, view, w.reshape(3, H, W))
    n_checked = 0
    for name in FIELDS3 + FIELDS4:
        a = sc[name]
        flat = a.reshape(-1)
        ga = g[name].reshape(-1)
        fd = np.zeros_like(ga)
        for k in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[k]))
            old = flat[k]
            flat[k] = old + h
            lp = loss(sc, view, w)
            flat[k] = old - h
            lm = loss(sc, view, w)
            flat[k] = old
            fd[k] = (lp - lm) / (2 * h)
        if flat.size:
            scale = max(1e-8, np.abs(fd).max())
            np.testing.assert_allclose(ga, fd, atol=rtol * scale * 10, rtol=1e-5, err_msg=name)
            n_checked += flat.size
    return n_checked


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradients_match_finite_differences(seed):
    sc, view = tiny_scene(seed)
    assert check_fd(sc, view) > 300


def test_gradients_with_clamped_jacobian():
    sc, view = tiny_scene(5, clamp_case=True)
    P = O.project(sc, view)
    i3 = sc["mean4"].shape[0]  # merged index of the first 3D Gaussian
    ux = (sc["mean3"][0, 0]) / sc["mean3"][0, 2]
    assert ux > 1.3 * view.W / (2 * view.fx) and P[i3]["visible"] == 1
    check_fd(sc, view)


def test_gradients_with_rotated_camera_and_background():
    sc, view = tiny_scene(3)
    ang = 0.1
    view.R = np.array([[np.cos(ang), 0, np.sin(ang)], [0, 1, 0], [-np.sin(ang), 0, np.cos(ang)]])
    view.T = np.array([0.05, -0.02, 0.1])
    view.bg = (0.2, 0.5, 0.9)
    check_fd(sc, view)


def test_dproj_is_the_2d_gradient():
    """The per-Gaussian 2D gradient (dproj) chained with finite differences of the
    projection reproduces the parameter gradient of the mean."""
    sc, view = tiny_scene(1)
    w = np.random.default_rng(3).normal(0, 1, (3, view.H, view.W))
    g = O.render_bwd(sc, view, w)
    n4 = sc["mean4"].shape[0]
    j = 0
    acc = np.zeros(3)
    for k in range(3):
        h = 1e-6
        sp = {kk: vv.copy() for kk, vv in sc.items()}
        sm = {kk: vv.copy() for kk, vv in sc.items()}
        sp["mean3"][j, k] += h
        sm["mean3"][j, k] -= h
        Pp, Pm = O.project(sp, view)[n4 + j], O.project(sm, view)[n4 + j]
        d = np.array([Pp["px"] - Pm["px"], Pp["py"] - Pm["py"], *(Pp["conic"] - Pm["conic"]),
                      Pp["alpha"] - Pm["alpha"], *(Pp["rgb"] - Pm["rgb"])]) / (2 * h)
        acc[k] = d @ g["dproj"][n4 + j]
    np.testing.assert_allclose(acc, g["mean3"][j], rtol=1e-6, atol=1e-9)


def test_gradients_with_time_dependent_colour():
    """The 4D colour with two time frequencies (blocks of 16 x 3 coefficients
    weighted by cos(2 pi n t)): every block's gradient, and all the others."""
    sc, view = tiny_scene(3, t=0.3)
    rng = np.random.default_rng(7)
    extra = rng.normal(0, 0.2, (sc["sh4"].shape[0], 32, 3))
    sc["sh4"] = np.concatenate([sc["sh4"], extra], 1)
    assert check_fd(sc, view) > 300
