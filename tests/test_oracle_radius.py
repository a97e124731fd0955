"""Pin of the oracle's support radius (Alg. 1 ProjGaussian3D/4D, the EWA
details of reading D5 inherited from 3DGS).

The oracle gives a projected Gaussian the radius ceil(3 sqrt(lam)) with
lam = mid + sqrt(max(0.1, mid^2 - det)) of the dilated 2D covariance
S' = J W Sigma W^T J^T + 0.3 I.  In terms of the eigenvalues l1 <= l2 of S'
(mid = (l1 + l2) / 2, mid^2 - det = ((l2 - l1) / 2)^2) that is the larger
eigenvalue l2, except that the half-gap (l2 - l1) / 2 is floored at sqrt(0.1)
for nearly isotropic footprints.  The radius decides the tile rectangle and so
which tiles list the Gaussian, which changes the image (the rectangle is part
of the support rule).

Nothing here uses the oracle's arithmetic: Sigma comes from scipy's rotation
of the quaternion, the Jacobian of the perspective map from central
differences, the eigenvalues from numpy's symmetric eigensolver, and the
isotropic case from its closed form ((f s / z)^2 + 0.3) I.  The cases are
chosen so that each plausible slip -- the smaller eigenvalue, 2 sigma instead
of 3, or no floor -- changes the radius of at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2505_13215_gb300 import scenes


def splats(means, log_scales, quats, opacity_logit=2.0):
    n = len(means)
    z = np.zeros
    return {"mean3": np.asarray(means, float), "log_scale3": np.asarray(log_scales, float),
            "quat3": np.asarray(quats, float), "opacity3": np.full(n, opacity_logit), "sh3": z((n, 16, 3)),
            "mean4": z((0, 4)), "log_scale4": z((0, 4)), "ql": z((0, 4)), "qr": z((0, 4)),
            "opacity4": z((0,)), "sh4": z((0, 16, 3))}


def dilated_cov2(view, mean, log_scale, quat):
    """S' of one 3D Gaussian by first principles: Sigma = R diag(exp 2s) R^T with
    R scipy's rotation of q = (w, x, y, z), pushed through the numerical Jacobian
    of x -> (fx x_c / z_c + cx, fy y_c / z_c + cy), plus 0.3 on the diagonal."""
    q = np.asarray(quat, float)
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = Rq @ np.diag(np.exp(2.0 * np.asarray(log_scale, float))) @ Rq.T
    Rc, Tc = np.asarray(view.R, float), np.asarray(view.T, float)

    def proj(x):
        xc = Rc @ x + Tc
        return np.array([view.fx * xc[0] / xc[2] + view.cx, view.fy * xc[1] / xc[2] + view.cy])

    m = np.asarray(mean, float)
    h = 1e-6
    J = np.stack([(proj(m + h * e) - proj(m - h * e)) / (2 * h) for e in np.eye(3)], 1)
    return J @ Sig @ J.T + 0.3 * np.eye(2)


def radius_readings(S2):
    """The radius of reading D5 and of the plausible slips, from eigvalsh(S')."""
    l1, l2 = np.linalg.eigvalsh(S2)
    mid, half_gap = 0.5 * (l1 + l2), 0.5 * (l2 - l1)
    lam = mid + max(math.sqrt(0.1), half_gap)
    return {"D5": math.ceil(3.0 * math.sqrt(lam)),
            "smaller_eigenvalue": math.ceil(3.0 * math.sqrt(mid - max(math.sqrt(0.1), half_gap))),
            "two_sigma": math.ceil(2.0 * math.sqrt(lam)),
            "no_floor": math.ceil(3.0 * math.sqrt(l2)),
            "_value": 3.0 * math.sqrt(lam), "_half_gap": half_gap}


def rotated_camera(angle=0.25, axis=(0.3, 1.0, -0.2), T=(0.2, -0.1, 0.4), W=256, H=192, fx=220.0, fy=200.0):
    ax = np.asarray(axis, float) / np.linalg.norm(axis)
    Rc = Rotation.from_rotvec(angle * ax).as_matrix()
    return scenes.View(R=Rc.astype(np.float64), T=np.asarray(T, float), fx=fx, fy=fy, cx=W / 2 + 3.0,
                       cy=H / 2 - 5.0, W=W, H=H, t=0.0)


def check_cases(view, means, log_scales, quats):
    P = O.project(splats(means, log_scales, quats), view)
    got, want = [], []
    for i in range(len(means)):
        assert P[i]["visible"] == 1, "case %d culled" % i
        r = radius_readings(dilated_cov2(view, means[i], log_scales[i], quats[i]))
        frac = r["_value"] - math.floor(r["_value"])
        assert 1e-6 < frac < 1 - 1e-6, "case %d sits on an integer radius; pick another" % i
        got.append(int(P[i]["radius"]))
        want.append(r)
    assert got == [r["D5"] for r in want], (got, [r["D5"] for r in want])
    return want


def test_isotropic_splat_closed_form_radius():
    """On the optical axis of an identity camera an isotropic Gaussian of scale s
    at depth z has S' = ((f s / z)^2 + 0.3) I: equal eigenvalues, so the floor
    decides and radius = ceil(3 sqrt((f s / z)^2 + 0.3 + sqrt(0.1)))."""
    f, z = 128.0, 4.0
    view = scenes.identity_view(128, 128, f, 0.0)
    var2d = [0.35, 0.65, 0.95, 1.7, 3.2, 6.5, 14.0, 40.0]  # (f s / z)^2
    ss = [math.sqrt(v) * z / f for v in var2d]
    means = [[0.0, 0.0, z]] * len(ss)
    P = O.project(splats(means, [[math.log(s)] * 3 for s in ss], [[1.0, 0, 0, 0]] * len(ss)), view)
    for p, v in zip(P, var2d):
        val = 3.0 * math.sqrt(v + 0.3 + math.sqrt(0.1))
        assert 1e-6 < val - math.floor(val) < 1 - 1e-6
        assert p["radius"] == math.ceil(val), (v, p["radius"], val)
    # the closed form separates the floor from its omission and 3 sigma from 2 sigma here
    assert any(math.ceil(3.0 * math.sqrt(v + 0.3)) != math.ceil(3.0 * math.sqrt(v + 0.3 + math.sqrt(0.1)))
               for v in var2d)
    assert any(math.ceil(2.0 * math.sqrt(v + 0.3 + math.sqrt(0.1))) !=
               math.ceil(3.0 * math.sqrt(v + 0.3 + math.sqrt(0.1))) for v in var2d)


def test_anisotropic_rotated_splats_take_the_larger_eigenvalue():
    """Strongly anisotropic Gaussians, randomly rotated, off axis, under a
    rotated and translated camera with fx != fy: the eigenvalue gap is far
    above the floor, so radius = ceil(3 sqrt(l2))."""
    rng = np.random.default_rng(11)
    view = rotated_camera()
    means, scales, quats = [], [], []
    Rc, Tc = np.asarray(view.R), np.asarray(view.T)
    while len(means) < 12:
        xc = np.array([rng.uniform(-0.25, 0.25), rng.uniform(-0.2, 0.2), 1.0]) * rng.uniform(2.0, 6.0)
        x = Rc.T @ (xc - Tc)
        ls = np.sort(rng.normal(-2.6, 0.2, 3)) + np.array([0.0, 0.6, 1.6])
        q = rng.standard_normal(4)
        r = radius_readings(dilated_cov2(view, x, ls, q))
        frac = r["_value"] - math.floor(r["_value"])
        if r["_half_gap"] < 4 * math.sqrt(0.1) or not 1e-3 < frac < 1 - 1e-3:
            continue
        means.append(x)
        scales.append(ls)
        quats.append(q)
    want = check_cases(view, means, scales, quats)
    assert all(r["D5"] == r["no_floor"] for r in want)  # the floor is inactive here
    assert any(r["smaller_eigenvalue"] != r["D5"] for r in want)
    assert any(r["two_sigma"] != r["D5"] for r in want)


def test_nearly_isotropic_splats_take_the_floor():
    """Footprints whose eigenvalues differ by less than 2 sqrt(0.1): the half-gap
    is floored, radius = ceil(3 sqrt(mid + sqrt(0.1))), which is not the larger
    eigenvalue's radius for some of them."""
    rng = np.random.default_rng(12)
    view = rotated_camera(angle=0.15)
    means, scales, quats = [], [], []
    Rc, Tc = np.asarray(view.R), np.asarray(view.T)
    while len(means) < 12:
        xc = np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 1.0]) * rng.uniform(3.0, 8.0)
        x = Rc.T @ (xc - Tc)
        base = rng.uniform(-4.2, -3.2)
        ls = base + rng.uniform(-0.05, 0.05, 3)
        q = rng.standard_normal(4)
        r = radius_readings(dilated_cov2(view, x, ls, q))
        frac = r["_value"] - math.floor(r["_value"])
        if r["_half_gap"] > 0.8 * math.sqrt(0.1) or not 1e-3 < frac < 1 - 1e-3:
            continue
        means.append(x)
        scales.append(ls)
        quats.append(q)
    want = check_cases(view, means, scales, quats)
    assert any(r["no_floor"] != r["D5"] for r in want)
    assert any(r["smaller_eigenvalue"] != r["D5"] for r in want)
    assert any(r["two_sigma"] != r["D5"] for r in want)


@pytest.mark.parametrize("seed", [21, 22])
def test_rectangle_follows_the_pinned_radius(seed):
    """The tile rectangle is [floor((p - r) / 16), ceil((p + r) / 16)) clipped to
    the grid, with r the radius pinned above and p the projected mean."""
    rng = np.random.default_rng(seed)
    view = rotated_camera(W=200, H=150)
    Rc, Tc = np.asarray(view.R), np.asarray(view.T)
    means, scales, quats = [], [], []
    for _ in range(16):
        xc = np.array([rng.uniform(-0.45, 0.45), rng.uniform(-0.35, 0.35), 1.0]) * rng.uniform(2.0, 5.0)
        means.append(Rc.T @ (xc - Tc))
        scales.append(rng.normal(-2.5, 0.5, 3))
        quats.append(rng.standard_normal(4))
    P = O.project(splats(means, scales, quats), view)
    TX, TY = math.ceil(view.W / 16), math.ceil(view.H / 16)
    for i, p in enumerate(P):
        if not p["visible"]:
            continue
        r = radius_readings(dilated_cov2(view, means[i], scales[i], quats[i]))["D5"]
        xc = Rc @ means[i] + Tc
        px, py = view.fx * xc[0] / xc[2] + view.cx, view.fy * xc[1] / xc[2] + view.cy
        rect = [min(max(math.floor((px - r) / 16), 0), TX), min(max(math.floor((py - r) / 16), 0), TY),
                min(max(math.ceil((px + r) / 16), 0), TX), min(max(math.ceil((py + r) / 16), 0), TY)]
        assert p["radius"] == r
        assert list(p["rect"]) == rect, (i, list(p["rect"]), rect)
