"""Pins of the oracle's densification (the 3DGS clone / split / prune rules
the paper adopts, Sec. 4.3): row accounting, copies, and the split children
distributed as the parent Gaussian -- the sample covariance of the children's
offsets M z over many draws approaches Sigma (Eq. 2 for a 3D Gaussian, the
4D covariance R S S^T R^T of Eq. 4 for a 4D one), which fixes M as a square
root of Sigma with the rotation the right way round."""
import numpy as np

import oracle as O
from paper_2505_13215_gb300 import scenes

RULE = dict(grad_threshold=2e-4, dense_scale=0.05, min_opacity=5e-3, split_shrink=np.log(1.6))


def _set(scene, four_d):
    a = scene.arrays()
    return {k: np.asarray(a[k], dtype=np.float64) for k in (O.FIELDS4 if four_d else O.FIELDS3)}


def test_row_accounting_and_copies():
    scene, _ = scenes.small_scene(seed=30, n3=400, n4=300)
    rng = np.random.default_rng(0)
    for four_d in (False, True):
        P = _set(scene, four_d)
        n = len(P["opacity4" if four_d else "opacity3"])
        m = {k: rng.normal(size=x.shape) for k, x in P.items()}
        v = {k: rng.uniform(size=x.shape) for k, x in P.items()}
        accum = rng.uniform(0, 6e-4, n)
        count = rng.integers(0, 3, n).astype(float)
        noise = rng.normal(size=(n, 2, 4 if four_d else 3))
        out, om, ov = O.densify_set(P, m, v, accum, count, noise, four_d=four_d, **RULE)
        o = P["opacity4" if four_d else "opacity3"]
        op = 1 / (1 + np.exp(-o))
        avg = np.where(count > 0, accum / np.maximum(count, 1), 0)
        ls = P["log_scale4" if four_d else "log_scale3"]
        big = np.exp(ls[:, :3].max(1)) > RULE["dense_scale"]
        alive = op >= RULE["min_opacity"]
        clone = alive & (avg >= 2e-4) & ~big
        split = alive & (avg >= 2e-4) & big
        keep = alive & ~split
        n_new = keep.sum() + clone.sum() + 2 * split.sum()
        for k in P:
            assert out[k].shape[0] == n_new
        kf = "sh4" if four_d else "sh3"
        # kept rows first, in order, with their moments; clones are exact copies with zero moments
        np.testing.assert_array_equal(out[kf][: keep.sum()], P[kf][keep])
        np.testing.assert_array_equal(om[kf][: keep.sum()], m[kf][keep])
        c0 = keep.sum()
        for k in P:
            np.testing.assert_array_equal(out[k][c0:c0 + clone.sum()], P[k][clone])
        assert not om[kf][c0:].any() and not ov[kf][c0:].any()
        # children: parent's fields, log-scales lowered by the shrink
        ch = out["log_scale4" if four_d else "log_scale3"][c0 + clone.sum():]
        np.testing.assert_allclose(ch[0::2], ls[split] - RULE["split_shrink"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(ch[1::2], ls[split] - RULE["split_shrink"], rtol=0, atol=1e-15)


def test_zero_draws_put_children_on_the_parent():
    scene, _ = scenes.small_scene(seed=31, n3=50, n4=50)
    for four_d in (False, True):
        P = _set(scene, four_d)
        n = 50
        P["opacity4" if four_d else "opacity3"][:] = 2.0
        P["log_scale4" if four_d else "log_scale3"][:] = np.log(0.2)  # all large: every one splits
        z = {k: np.zeros_like(x) for k, x in P.items()}
        out, _, _ = O.densify_set(P, z, z, np.ones(n), np.ones(n), np.zeros((n, 2, 4 if four_d else 3)),
                                  four_d=four_d, **RULE)
        mu = P["mean4" if four_d else "mean3"]
        np.testing.assert_array_equal(out["mean4" if four_d else "mean3"][0::2], mu)
        np.testing.assert_array_equal(out["mean4" if four_d else "mean3"][1::2], mu)


def test_children_follow_the_parent_distribution():
    rng = np.random.default_rng(3)
    draws = 40000
    q3 = rng.normal(size=4)
    s3 = np.array([np.log(0.3), np.log(0.1), np.log(0.05)])
    ql, qr = rng.normal(size=4), rng.normal(size=4)
    s4 = np.array([np.log(0.3), np.log(0.1), np.log(0.05), np.log(0.2)])
    for four_d, Sigma in ((False, O.cov3(q3, s3)), (True, O.cov4(ql, qr, s4))):
        d = 4 if four_d else 3
        P = ({"mean4": np.zeros((1, 4)), "log_scale4": s4[None], "ql": ql[None], "qr": qr[None],
              "opacity4": np.array([3.0]), "sh4": np.zeros((1, 16, 3))} if four_d else
             {"mean3": np.zeros((1, 3)), "log_scale3": s3[None], "quat3": q3[None], "opacity3": np.array([3.0]),
              "sh3": np.zeros((1, 16, 3))})
        z = {k: np.zeros_like(x) for k, x in P.items()}
        # the map from a draw to a child's offset, read column by column with unit draws
        eye = np.eye(d)
        cols = []
        for j in range(d):
            nz = np.zeros((1, 2, d))
            nz[0, 0] = eye[j]
            out, _, _ = O.densify_set(P, z, z, np.ones(1), np.ones(1), nz, four_d=four_d, **RULE)
            cols.append(out["mean4" if four_d else "mean3"][0])
        M = np.stack(cols, 1)
        # linear in the draw: a random draw lands where M says
        zr = rng.normal(size=(1, 2, d))
        out, _, _ = O.densify_set(P, z, z, np.ones(1), np.ones(1), zr, four_d=four_d, **RULE)
        np.testing.assert_allclose(out["mean4" if four_d else "mean3"][1], M @ zr[0, 1], rtol=1e-12, atol=1e-14)
        # children distributed as the parent: offsets M z with z ~ N(0, I) have covariance M M^T = Sigma
        np.testing.assert_allclose(M @ M.T, Sigma, rtol=1e-9, atol=1e-12)
        emp = np.cov((rng.normal(size=(draws, d)) @ M.T).T)
        np.testing.assert_allclose(emp, Sigma, atol=0.03 * np.abs(Sigma).max())


def test_stats_are_ndc_gradient_norms():
    g = np.array([[1.0, 0.0], [0.0, 2.0], [3.0, 4.0]])
    acc, cnt = O.densify_stats(g, [True, True, False], W=200, H=100)
    np.testing.assert_allclose(acc, [100.0, 100.0, 0.0])
    np.testing.assert_array_equal(cnt, [1, 1, 0])
