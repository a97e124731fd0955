"""Pins of the oracle's Adam step against properties the algorithm fixes
(Kingma and Ba, 2015): a constant gradient moves every coordinate by exactly
lr g / (|g| + eps) per step (the bias corrections make m_hat = g and
v_hat = g^2 from the first step on); with eps = 0 the update is invariant to a
positive scaling of the gradient and odd in its sign; the moments are
exponential moving averages with the stated weights."""
import numpy as np

import oracle as O


def test_constant_gradient_moves_by_lr_sign_each_step():
    rng = np.random.default_rng(0)
    g = rng.normal(size=50)
    p0 = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 8):
        p, m, v = O.adam_step(p, m, v, g, t, lr, 0.9, 0.999, eps)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)


def test_scale_invariance_and_sign_symmetry_without_eps():
    rng = np.random.default_rng(1)
    gs = [rng.normal(size=20) for _ in range(5)]
    p0 = rng.normal(size=20)

    def run(scale):
        p, m, v = p0.copy(), np.zeros(20), np.zeros(20)
        for t, g in enumerate(gs, 1):
            p, m, v = O.adam_step(p, m, v, scale * g, t, 0.01, 0.9, 0.99, 0.0)
        return p - p0

    np.testing.assert_allclose(run(1.0), run(37.0), rtol=1e-12)
    np.testing.assert_allclose(run(1.0), -run(-1.0), rtol=1e-12)


def test_moments_are_exponential_averages():
    rng = np.random.default_rng(2)
    gs = rng.normal(size=(6, 4))
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t, g in enumerate(gs, 1):
        p, m, v = O.adam_step(p, m, v, g, t, 0.1, 0.8, 0.95, 1e-8)
    w1 = np.array([0.2 * 0.8 ** (6 - k) for k in range(1, 7)])
    w2 = np.array([0.05 * 0.95 ** (6 - k) for k in range(1, 7)])
    np.testing.assert_allclose(m, (w1[:, None] * gs).sum(0), rtol=1e-12)
    np.testing.assert_allclose(v, (w2[:, None] * gs * gs).sum(0), rtol=1e-12)


def test_per_coordinate_step_sizes():
    g = np.array([1.0, -2.0, 0.5])
    lr = np.array([1e-3, 1e-2, 1e-1])
    p, _, _ = O.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr, 0.9, 0.999, 0.0)
    np.testing.assert_allclose(p, -lr * np.sign(g), rtol=1e-12)
