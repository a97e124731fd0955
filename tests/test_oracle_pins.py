"""Pins of the FP64 oracle to facts outside itself: quaternion algebra, closed
forms of Gaussian conditioning, brute-force marginalisation, analytic splat
footprints, sphere quadrature and central finite differences.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_13215_gb300 import scenes


def qmul(p, q):
    """Hamilton product of quaternions (w, x, y, z)."""
    a1, b1, c1, d1 = p
    a2, b2, c2, d2 = q
    return np.array([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2,
                     a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                     a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2,
                     a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2])


def qconj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])


def unit(rng, n=4):
    q = rng.standard_normal(n)
    return q / np.linalg.norm(q)


RNG = np.random.default_rng(1234)
QUAT_PAIRS = [(unit(RNG) * RNG.uniform(0.5, 2.0), unit(RNG) * RNG.uniform(0.5, 2.0)) for _ in range(20)]


# ---------------------------------------------------------------------------
# Eq. 4: the 4D rotation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ql,qr", QUAT_PAIRS)
def test_rot4_orthonormal(ql, qr):
    R = O.rot4(ql, qr)
    np.testing.assert_allclose(R @ R.T, np.eye(4), atol=1e-13)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12


@pytest.mark.parametrize("ql,qr", QUAT_PAIRS[:8])
def test_rot4_is_left_times_right_quaternion_multiplication(ql, qr):
    """R_l and R_r of Eq. 4 are the matrices of x -> q_l x and x -> x q_r, so R x = q_l x q_r."""
    a, b = ql / np.linalg.norm(ql), qr / np.linalg.norm(qr)
    R = O.rot4(ql, qr)
    for _ in range(4):
        x = RNG.standard_normal(4)
        np.testing.assert_allclose(R @ x, qmul(qmul(a, x), b), atol=1e-13)


def k_fixing_qr(ql):
    """The right quaternion that makes R_4D block diagonal (Eq. 8): q_l k q_r = k."""
    k = np.array([0.0, 0.0, 0.0, 1.0])
    a = ql / np.linalg.norm(ql)
    return qmul(qmul(qconj(k), qconj(a)), k)


@pytest.mark.parametrize("ql,_", QUAT_PAIRS[:6])
def test_rot4_block_diagonal_case(ql, _):
    R = O.rot4(ql, k_fixing_qr(ql))
    e4 = np.array([0, 0, 0, 1.0])
    np.testing.assert_allclose(R[3], e4, atol=1e-13)
    np.testing.assert_allclose(R[:, 3], e4, atol=1e-13)
    R3 = R[:3, :3]
    np.testing.assert_allclose(R3 @ R3.T, np.eye(3), atol=1e-13)


# ---------------------------------------------------------------------------
# Eq. 2 and the 3D rotation that Eq. 9 inverts
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q,_", QUAT_PAIRS[:6])
def test_quat_to_R3_rotates_like_q_v_qconj(q, _):
    R = O.quat_to_R3(q)
    qn = q / np.linalg.norm(q)
    for _ in range(3):
        v = RNG.standard_normal(3)
        rv = qmul(qmul(qn, np.r_[0.0, v]), qconj(qn))
        np.testing.assert_allclose(R @ v, rv[1:], atol=1e-13)


@pytest.mark.parametrize("q,_", QUAT_PAIRS[:6])
def test_cov3_spectrum(q, _):
    s = RNG.normal(-1, 0.5, 3)
    S = O.cov3(q, s)
    R = O.quat_to_R3(q)
    np.testing.assert_allclose(S, S.T, atol=1e-15)
    for k in range(3):  # columns of R are eigenvectors with eigenvalue exp(2 s_k)
        np.testing.assert_allclose(S @ R[:, k], np.exp(2 * s[k]) * R[:, k], rtol=1e-12, atol=1e-14)


def test_cov4_is_rotated_scale():
    ql, qr = QUAT_PAIRS[0]
    s = np.array([-1.0, -0.5, -2.0, 0.3])
    S = O.cov4(ql, qr, s)
    R = O.rot4(ql, qr)
    w, V = np.linalg.eigh(S)
    np.testing.assert_allclose(np.sort(w), np.sort(np.exp(2 * s)), rtol=1e-12)
    for k in range(4):
        np.testing.assert_allclose(S @ R[:, k], np.exp(2 * s[k]) * R[:, k], rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# Eq. 5/6 and the temporal factor (reading D1)
# ---------------------------------------------------------------------------

def gauss_unnorm(x, mu, S):
    d = x - mu
    return np.exp(-0.5 * d @ np.linalg.solve(S, d))


@pytest.mark.parametrize("ql,qr", QUAT_PAIRS[:6])
def test_slice_factorisation_identity(ql, qr):
    """G4(x, t) = p(t) G3(x; mu_{x|t}, Sigma_{x|t}) pointwise: the conditional plus
    the unnormalised marginal reproduce the 4D Gaussian exactly."""
    s = RNG.normal(-1.0, 0.4, 4)
    m4 = RNG.standard_normal(4)
    S4 = O.cov4(ql, qr, s)
    for t in (m4[3] - 0.3, m4[3], m4[3] + 0.7):
        mu, S3, p = O.slice(m4, S4, t)
        for _ in range(5):
            x = mu + RNG.normal(0, 0.5, 3)
            g4 = gauss_unnorm(np.r_[x, t], m4, S4)
            g3 = gauss_unnorm(x, mu, S3)
            assert abs(g4 - p * g3) <= 1e-12 * max(1.0, g4)


def test_slice_brute_force_marginalisation():
    """Moments of G4(., t) on a dense grid match mu_{x|t}, Sigma_{x|t}, and
    integral(G4(., t)) / integral(G3(.; mu, Sigma_{x|t})) = p(t)."""
    ql, qr = QUAT_PAIRS[3]
    s = np.array([-0.6, -0.9, -0.4, -0.5])
    m4 = np.array([0.1, -0.2, 0.3, 0.4])
    S4 = O.cov4(ql, qr, s)
    t = 0.75
    mu, S3, p = O.slice(m4, S4, t)
    n = 72
    half = 6.0 * np.sqrt(np.max(np.diag(S3)))
    ax = [np.linspace(mu[k] - half, mu[k] + half, n) for k in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    P = np.stack([X, Y, Z, np.full_like(X, t)], -1).reshape(-1, 4)
    Si = np.linalg.inv(S4)
    D = P - m4
    g = np.exp(-0.5 * np.einsum("ni,ij,nj->n", D, Si, D))
    w = g.sum()
    m1 = (g[:, None] * P[:, :3]).sum(0) / w
    C = ((g[:, None, None] * (P[:, :3] - m1)[:, :, None] * (P[:, :3] - m1)[:, None, :]).sum(0)) / w
    np.testing.assert_allclose(m1, mu, atol=1e-6)
    np.testing.assert_allclose(C, S3, rtol=1e-3, atol=1e-6)
    S3i = np.linalg.inv(S3)
    D3 = P[:, :3] - mu
    g3 = np.exp(-0.5 * np.einsum("ni,ij,nj->n", D3, S3i, D3))
    assert abs(w / g3.sum() - p) < 1e-9
    assert 0.0 < p < 1.0


def test_slice_zero_space_time_covariance():
    """Eq. 8 ideal case: R_4D block diagonal gives mu_{x|t} = mu_x, Sigma_{x|t} =
    R_3D S^2 R_3D^T and p(t) = exp(-(t - mu_t)^2 / (2 exp(2 s_t)))."""
    ql = QUAT_PAIRS[5][0]
    qr = k_fixing_qr(ql)
    s = np.array([-1.0, -1.5, -0.7, -1.2])
    m4 = np.array([0.5, 0.2, 3.0, 0.4])
    S4 = O.cov4(ql, qr, s)
    R3 = O.rot4(ql, qr)[:3, :3]
    for t in (0.4, 0.55, 0.9):
        mu, S3, p = O.slice(m4, S4, t)
        np.testing.assert_allclose(mu, m4[:3], atol=1e-14)
        np.testing.assert_allclose(S3, R3 @ np.diag(np.exp(2 * s[:3])) @ R3.T, atol=1e-14)
        assert abs(p - math.exp(-0.5 * (t - 0.4) ** 2 / math.exp(2 * s[3]))) < 1e-14


# ---------------------------------------------------------------------------
# Eq. 9 and the conversion of Sec. 4.2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q,_", QUAT_PAIRS[:10])
def test_eq9_round_trip(q, _):
    qn = q / np.linalg.norm(q)
    qn = qn if qn[0] >= 0 else -qn
    np.testing.assert_allclose(O.matrix_to_quat(O.quat_to_R3(q)), qn, atol=1e-12)


@pytest.mark.parametrize("axis", [np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0]),
                                  np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])])
def test_eq9_half_turn_branches(axis):
    """Rotations by (nearly) pi have 1 + tr(R) ~ 0 where the printed formula divides
    by ~0; every largest-diagonal branch must still invert the rotation."""
    for ang in (math.pi, math.pi - 1e-3):
        q = np.r_[math.cos(ang / 2), math.sin(ang / 2) * axis]
        got = O.matrix_to_quat(O.quat_to_R3(q))
        np.testing.assert_allclose(O.quat_to_R3(got), O.quat_to_R3(q), atol=1e-12)
        assert got[0] >= 0 and abs(np.linalg.norm(got) - 1) < 1e-14


def test_eq9_literal_values():
    """The printed formula on a hand-made rotation: 90 degrees about z."""
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    # w = sqrt(1 + 1)/2, z = (R21 - R12) / (4 w) = 2 / (4 w)
    w = 0.5 * math.sqrt(2.0)
    np.testing.assert_allclose(O.matrix_to_quat(R), [w, 0, 0, 2 / (4 * w)], atol=1e-15)


def test_convert_classification_and_fields():
    scene, _ = scenes.small_scene(seed=3, n3=5, n4=40)
    tau = 0.14
    moved, app, keep = O.convert(scene, tau)
    st = np.exp(scene.log_scale4[:, 3].astype(np.float64))
    np.testing.assert_array_equal(moved, st > tau)
    idx = np.nonzero(moved)[0]
    np.testing.assert_array_equal(keep, np.nonzero(~moved)[0])
    np.testing.assert_array_equal(app["mean3"], scene.mean4[idx, :3])
    np.testing.assert_array_equal(app["log_scale3"], scene.log_scale4[idx, :3])
    np.testing.assert_array_equal(app["opacity3"], scene.opacity4[idx])
    np.testing.assert_array_equal(app["sh3"], scene.sh4[idx])
    for j, i in enumerate(idx):
        R3 = O.rot4(scene.ql[i], scene.qr[i])[:3, :3]
        q = app["quat3"][j]
        assert abs(np.linalg.norm(q) - 1) < 1e-12 and q[0] >= 0
        # Eq. 9 applied to the (generally not orthonormal) top-left block
        tr = np.trace(R3)
        if 1 + tr > 1e-2:
            w = 0.5 * math.sqrt(1 + tr)
            raw = np.array([w, (R3[2, 1] - R3[1, 2]) / (4 * w), (R3[0, 2] - R3[2, 0]) / (4 * w),
                            (R3[1, 0] - R3[0, 1]) / (4 * w)])
            np.testing.assert_allclose(q, raw / np.linalg.norm(raw), atol=1e-12)


# ---------------------------------------------------------------------------
# Spherical harmonics (reading D8)
# ---------------------------------------------------------------------------

def test_sh_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phis = np.arange(nphi) * 2 * math.pi / nphi
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            Y = O.sh_basis([r * math.cos(ph), r * math.sin(ph), z])
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_low_order_closed_forms():
    """Degree 0 is the constant 1/(2 sqrt(pi)); degree 1 is sqrt(3/(4 pi)) (-y, z, -x)
    (Condon-Shortley phase, m = -1, 0, 1)."""
    for _ in range(5):
        d = unit(RNG, 3)
        Y = O.sh_basis(d)
        assert abs(Y[0] - 0.5 / math.sqrt(math.pi)) < 1e-15
        c1 = math.sqrt(3 / (4 * math.pi))
        np.testing.assert_allclose(Y[1:4], c1 * np.array([-d[1], d[2], -d[0]]), atol=1e-15)
        # Y_2^0 = sqrt(5/(16 pi)) (3 z^2 - 1)
        assert abs(Y[6] - math.sqrt(5 / (16 * math.pi)) * (3 * d[2] ** 2 - 1)) < 1e-14


def test_sh_gradient_tangential_part_matches_fd():
    for _ in range(5):
        d = unit(RNG, 3)
        Y, dY = O.sh_basis(d, with_grad=True)
        for _ in range(2):
            tvec = np.cross(d, unit(RNG, 3))
            tvec /= np.linalg.norm(tvec)
            h = 1e-6
            dp = (d + h * tvec) / np.linalg.norm(d + h * tvec)
            dm = (d - h * tvec) / np.linalg.norm(d - h * tvec)
            fd = (O.sh_basis(dp) - O.sh_basis(dm)) / (2 * h)
            np.testing.assert_allclose(dY @ tvec, fd, atol=1e-7)


# ---------------------------------------------------------------------------
# EWA projection and compositing: analytic footprints
# ---------------------------------------------------------------------------

def one_splat(mean, log_scale, opacity_logit, dc=(0.0, 0.0, 0.0), quat=(1.0, 0, 0, 0), sh_extra=None):
    sh = np.zeros((1, 16, 3))
    sh[0, 0] = dc
    if sh_extra is not None:
        sh[0] += sh_extra
    z = np.zeros
    return {"mean3": np.array([mean], float), "log_scale3": np.array([log_scale], float),
            "quat3": np.array([quat], float), "opacity3": np.array([opacity_logit], float), "sh3": sh,
            "mean4": z((0, 4)), "log_scale4": z((0, 4)), "ql": z((0, 4)), "qr": z((0, 4)),
            "opacity4": z((0,)), "sh4": z((0, 16, 3))}


def cat(*ss):
    return {k: np.concatenate([s[k] for s in ss], 0) for k in ss[0]}


def test_isotropic_splat_analytic_footprint():
    f, z, s = 128.0, 4.0, math.exp(-3.0)
    view = scenes.identity_view(128, 128, f, 0.0)
    sc = one_splat([0.0, 0.0, z], [math.log(s)] * 3, 0.8, dc=(0.3, -0.2, 1.1))
    P = O.project(sc, view)[0]
    var = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(P["conic"], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
    assert P["px"] == 64.0 and P["py"] == 64.0 and P["depth"] == z
    sig = 1 / (1 + math.exp(-0.8))
    c = np.array([0.3, -0.2, 1.1]) * 0.5 / math.sqrt(math.pi) + 0.5
    c = np.maximum(c, 0.0)
    r = O.render(sc, view)
    img = r["rgb"].reshape(3, 128, 128)
    x0, y0, x1, y1 = P["rect"]
    for (u, v) in [(64, 64), (65, 64), (66, 67), (60, 70), (64, 58)]:
        a = min(0.99, sig * math.exp(-((u - 64) ** 2 + (v - 64) ** 2) / (2 * var)))
        inside = x0 <= u // 16 < x1 and y0 <= v // 16 < y1
        expect = c * a if (a >= 1 / 255 and inside) else np.zeros(3)
        np.testing.assert_allclose(img[:, v, u], expect, atol=1e-14)
        if a >= 1 / 255 and inside:
            assert abs(r["T"].reshape(128, 128)[v, u] - (1 - a)) < 1e-14


def test_rect_bounds_the_support():
    """Nothing is drawn outside the tile rectangle and the rectangle holds the
    disc of the radius."""
    view = scenes.identity_view(128, 128, 128.0, 0.0)
    sc = one_splat([0.3, -0.2, 3.0], [-2.0, -2.6, -2.2], 2.0, dc=(1.0, 1.0, 1.0), quat=(0.9, 0.1, -0.3, 0.2))
    P = O.project(sc, view)[0]
    r = O.render(sc, view)
    img = r["rgb"].reshape(3, 128, 128).sum(0)
    x0, y0, x1, y1 = P["rect"]
    mask = np.zeros((128, 128), bool)
    mask[y0 * 16: y1 * 16, x0 * 16: x1 * 16] = True
    assert np.all(img[~mask] == 0.0)
    assert img[mask].max() > 0
    R = P["radius"]
    assert x0 * 16 <= P["px"] - R and P["px"] + R <= x1 * 16
    assert y0 * 16 <= P["py"] - R and P["py"] + R <= y1 * 16


def test_ewa_matches_numerical_linearisation():
    """Off axis and under a rotated, translated camera, the 2D covariance is the
    first-order push-forward of Sigma through the perspective map (plus the 0.3
    px^2 dilation) and the 2D mean is the projected mean."""
    ax = np.array([0.2, 1.0, -0.4]) / np.linalg.norm([0.2, 1.0, -0.4])
    ang = 0.3
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rc = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    Tc = np.array([0.3, -0.1, 0.5])
    view = scenes.View(R=Rc, T=Tc, fx=140.0, fy=120.0, cx=60.0, cy=70.0, W=128, H=128, t=0.0)
    mean = np.array([0.4, 0.3, 3.5])
    q = np.array([0.8, 0.3, -0.2, 0.4])
    ls = np.array([-2.0, -2.5, -1.8])
    P = O.project(one_splat(mean, ls, 1.0, quat=q), view)[0]
    Sig = O.cov3(q, ls)

    def proj(x):
        xc = Rc @ x + Tc
        return np.array([140.0 * xc[0] / xc[2] + 60.0, 120.0 * xc[1] / xc[2] + 70.0])

    h = 1e-6
    Jn = np.stack([(proj(mean + h * e) - proj(mean - h * e)) / (2 * h) for e in np.eye(3)], 1)
    S2 = Jn @ Sig @ Jn.T + 0.3 * np.eye(2)
    conic = np.linalg.inv(S2)
    np.testing.assert_allclose(P["conic"], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-7)
    np.testing.assert_allclose([P["px"], P["py"]], proj(mean), rtol=1e-14)
    np.testing.assert_allclose(P["depth"], (Rc @ mean + Tc)[2], rtol=1e-14)


def test_render_invariant_under_rigid_motion():
    """Moving the camera by (R, T) equals moving the world by (R, T) under an identity
    camera (view-independent colour)."""
    scene, _ = scenes.small_scene(seed=7, n3=40, n4=0)
    sc = scene.arrays()
    sc["sh3"] = sc["sh3"].astype(np.float64).copy()
    sc["sh3"][:, 1:] = 0.0
    ax = np.array([1.0, -0.3, 0.2]) / np.linalg.norm([1.0, -0.3, 0.2])
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rc = np.eye(3) + math.sin(0.2) * K + (1 - math.cos(0.2)) * K @ K
    Tc = np.array([0.1, 0.2, 0.3])
    cam = scenes.View(R=Rc, T=Tc, fx=128.0, fy=128.0, cx=64.0, cy=64.0, W=64, H=64, t=0.0)
    a = O.render(sc, cam)
    # world-moved scene: means R mu + T, rotations q_c * q
    qc = O.matrix_to_quat(Rc)
    moved = dict(sc)
    moved["mean3"] = (sc["mean3"].astype(np.float64) @ Rc.T) + Tc
    moved["quat3"] = np.stack([qmul(qc, q / np.linalg.norm(q)) for q in sc["quat3"].astype(np.float64)])
    b = O.render(moved, scenes.View(R=np.eye(3), T=np.zeros(3), fx=128.0, fy=128.0, cx=64.0, cy=64.0,
                                    W=64, H=64, t=0.0))
    ok = (a["margin_fwd"] > 1e-6) & (b["margin_fwd"] > 1e-6)
    np.testing.assert_allclose(a["rgb"][:, ok], b["rgb"][:, ok], atol=1e-10)
    assert ok.mean() > 0.95


def test_sh_colour_uses_view_direction():
    """Only Y_1^0 set: colour = 0.5 + k sqrt(3/(4 pi)) d_z with d the unit vector
    from the camera centre -R^T T to the mean."""
    Tc = np.array([0.4, -0.3, 0.2])
    view = scenes.View(R=np.eye(3), T=Tc, fx=128.0, fy=128.0, cx=64.0, cy=64.0, W=128, H=128, t=0.0)
    extra = np.zeros((16, 3))
    extra[2] = [0.5, -0.7, 0.2]
    mean = np.array([0.5, 0.4, 3.0])
    P = O.project(one_splat(mean, [-2.0] * 3, 1.0, sh_extra=extra), view)[0]
    d = mean - (-Tc)
    d /= np.linalg.norm(d)
    expect = np.maximum(0.5 + extra[2] * math.sqrt(3 / (4 * math.pi)) * d[2], 0)
    np.testing.assert_allclose(P["rgb"], expect, atol=1e-14)


def test_two_splats_order_by_depth():
    view = scenes.identity_view(64, 64, 64.0, 0.0)
    near = one_splat([0.0, 0.0, 2.0], [-1.5] * 3, 0.5, dc=(1.0, 0.0, 0.0))
    far = one_splat([0.0, 0.0, 3.0], [-1.2] * 3, 1.5, dc=(0.0, 1.0, 0.0))
    r1 = O.render(cat(near, far), view)
    r2 = O.render(cat(far, near), view)
    np.testing.assert_allclose(r1["rgb"], r2["rgb"], atol=1e-15)  # index order does not matter
    Pn = O.project(near, view)[0]
    Pf = O.project(far, view)[0]
    u = v = 32
    an = min(0.99, Pn["alpha"])
    af = min(0.99, Pf["alpha"])
    c1 = Pn["rgb"] * an + Pf["rgb"] * af * (1 - an)
    np.testing.assert_allclose(r1["rgb"].reshape(3, 64, 64)[:, v, u], c1, atol=1e-14)


def test_depth_key_is_fp32_then_merged_index():
    """Reading D6: the sort key holds the depth as an FP32 number (Alg. 1 sorts
    tile|depth keys), so two splats whose depths round to the same FP32 value are
    composited in merged-index order even when FP64 puts them the other way."""
    th = 1e-3
    view = scenes.identity_view(64, 64, 64.0, 0.0)
    R = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    view = dataclasses.replace(view, R=R)
    a = one_splat([0.0, 0.0, 3.0], [-1.5] * 3, 1.0, dc=(1.0, 0.0, 0.0))
    b = one_splat([-1e-5, 0.0, 3.0], [-1.5] * 3, 1.0, dc=(0.0, 1.0, 0.0))  # 1e-8 farther
    Pa, Pb = O.project(a, view)[0], O.project(b, view)[0]
    assert Pb["depth"] > Pa["depth"] and np.float32(Pb["depth"]) == np.float32(Pa["depth"])
    u, v = int(Pa["px"]), int(Pa["py"])
    pix = [v * 64 + u]
    alpha = {}
    for name, P in (("a", Pa), ("b", Pb)):
        dx, dy = P["px"] - u, P["py"] - v
        ca, cb, cc = P["conic"]
        alpha[name] = min(0.99, P["alpha"] * math.exp(-0.5 * (ca * dx * dx + cc * dy * dy) - cb * dx * dy))
    for first, second, scene in (("b", "a", cat(b, a)), ("a", "b", cat(a, b))):
        P = {"a": Pa, "b": Pb}
        want = P[first]["rgb"] * alpha[first] + P[second]["rgb"] * alpha[second] * (1 - alpha[first])
        got = O.render(scene, view, pixels=pix)["rgb"][:, 0]
        np.testing.assert_allclose(got, want, atol=1e-14)


def test_transmittance_stop_and_bounds():
    """Final T stays in [1e-4, 1], composite colour <= (1 - T) max c for a black
    background, and 'last' is where the walk ends: a stop needs T (1 - alpha) <
    1e-4 with alpha <= 0.99, i.e. T < 0.01, so a pixel that kept T >= 0.01 walked
    its whole tile list, and one that stopped early ended below 0.01."""
    scene, views = scenes.small_scene(seed=0)
    v = views[0]
    r = O.render(scene, v)
    P = O.project(scene, v)
    cmax = P["rgb"][P["visible"] == 1].max(0)
    assert r["T"].min() >= 1e-4 and r["T"].max() <= 1.0
    assert np.all(r["rgb"] <= (1 - r["T"])[None] * cmax[:, None] + 1e-12)
    TX, TY = (v.W + 15) // 16, (v.H + 15) // 16
    length = np.array([[len(O.tile_list(scene, v, tx, ty)) for tx in range(TX)] for ty in range(TY)])
    yy, xx = np.divmod(np.arange(v.W * v.H), v.W)
    m = length[yy // 16, xx // 16]
    assert np.all(r["last"] <= m)
    assert np.all(r["last"][r["T"] >= 0.01] == m[r["T"] >= 0.01])
    assert np.all(r["T"][r["last"] < m] < 0.01)
    assert np.any(r["last"] < m) and np.any(r["T"] >= 0.01)


@pytest.mark.parametrize("seed,n3,n4,tiles", [(4, 300, 100, [(3, 3), (4, 2), (0, 7)]),
                                              (0, 3072, 1024, [(3, 4), (4, 3)])])
def test_transmittance_monotone_along_list(seed, n3, n4, tiles):
    """Walk a pixel's tile list by hand: T never rises, the final T is the
    renderer's, and the walk ends where 'last' says (the dense scene's pixels
    saturate and stop early)."""
    scene, views = scenes.small_scene(seed=seed, n3=n3, n4=n4)
    v = views[0]
    P = O.project(scene, v)
    stopped = 0
    for (tx, ty) in tiles:
        ids = O.tile_list(scene, v, tx, ty)
        assert np.all(np.diff(P["depth"][ids].astype(np.float32)) >= 0)
        u, vv = tx * 16 + 5, ty * 16 + 9
        T, end = 1.0, len(ids)
        for j, i in enumerate(ids):
            p = P[i]
            dx, dy = p["px"] - u, p["py"] - vv
            a, b, c = p["conic"]
            pw = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
            al = min(0.99, p["alpha"] * math.exp(pw))
            if pw > 0 or al < 1 / 255:
                continue
            if T * (1 - al) < 1e-4:
                end = j
                break
            assert T * (1 - al) <= T
            T *= 1 - al
        r = O.render(scene, v, pixels=[vv * v.W + u])
        assert abs(T - r["T"][0]) < 1e-14
        assert r["last"][0] == end
        stopped += end < len(ids)
    assert stopped == (len(tiles) if n3 > 1000 else 0)


def test_stable_sort_against_numpy():
    rng = np.random.default_rng(5)
    k = rng.integers(0, 50, 2000).astype(np.uint64) << np.uint64(32) | rng.integers(0, 4, 2000).astype(np.uint64)
    np.testing.assert_array_equal(O.stable_sort_u64(k), np.argsort(k, kind="stable"))
    assert O.stable_sort_u64(np.zeros(0, np.uint64)).shape == (0,)


def test_temporal_cull_of_4d():
    """A 4D Gaussian far from its time centre has alpha_max = sigmoid(o) p(t) < 1/255 and is culled."""
    s, _ = scenes.small_scene(seed=1, n3=0, n4=1)
    sc = s.arrays()
    sc["mean4"] = np.array([[0.0, 0.0, 3.0, 0.0]], np.float64)
    sc["log_scale4"] = np.array([[-2.0, -2.0, -2.0, -3.0]])
    v = scenes.identity_view(64, 64, 64.0, 0.0)
    assert O.project(sc, v)[0]["visible"] == 1
    v.t = 0.9
    P = O.project(sc, v)[0]
    assert P["visible"] == 0 and P["alpha"] < 1 / 255


# ---------------------------------------------------------------------------
# Eq. 8 ideal case end to end: 4D == converted 3D
# ---------------------------------------------------------------------------

def test_ideal_4d_renders_like_its_3d_conversion():
    rng = np.random.default_rng(11)
    n = 30
    base, _ = scenes.small_scene(seed=11, n3=0, n4=n)
    sc = {k: v.astype(np.float64) for k, v in base.arrays().items()}
    sc["qr"] = np.stack([k_fixing_qr(q) for q in sc["ql"]])
    sc["log_scale4"][:, 3] = rng.normal(0.0, 0.3, n)
    view = scenes.identity_view(128, 128, 128.0, 0.45)
    a = O.render(sc, view)
    # 3D equivalent: Eq. 9 rotation, opacity sigmoid(o') = sigmoid(o) p(t)
    moved, app, _ = O.convert(sc, 0.0)
    assert moved.all()
    pt = np.exp(-0.5 * (0.45 - sc["mean4"][:, 3]) ** 2 / np.exp(2 * sc["log_scale4"][:, 3]))
    sg = pt / (1 + np.exp(-sc["opacity4"]))
    z = np.zeros
    sc3 = {"mean3": app["mean3"], "log_scale3": app["log_scale3"], "quat3": app["quat3"],
           "opacity3": np.log(sg / (1 - sg)), "sh3": app["sh3"], "mean4": z((0, 4)), "log_scale4": z((0, 4)),
           "ql": z((0, 4)), "qr": z((0, 4)), "opacity4": z((0,)), "sh4": z((0, 16, 3))}
    b = O.render(sc3, view)
    ok = (a["margin_fwd"] > 1e-6) & (b["margin_fwd"] > 1e-6)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(a["rgb"][:, ok], b["rgb"][:, ok], atol=1e-10)
    # at t = mu_t the temporal factor is exactly 1
    i = 0
    v2 = scenes.identity_view(128, 128, 128.0, float(sc["mean4"][i, 3]))
    P4 = O.project(sc, v2)[i]
    assert abs(P4["alpha"] - 1 / (1 + math.exp(-sc["opacity4"][i]))) < 1e-15
