"""Pins of the 4D time-dependent colour (4D spherindrical harmonics, the
colour model Sec. 3.2 defers to 4DGS for): colour(d, t) = max(0, 0.5 +
sum_n cos(2 pi n t) sum_k c_nk Y_k(d)).  Cases where the cosines take known
values reduce it to the plain degree-3 SH colour of a combined coefficient
block; over a full period the higher frequencies average out."""
import dataclasses

import numpy as np

import oracle as O
from paper_2505_13215_gb300 import scenes


def _scene(n_time, seed=0):
    scene, views = scenes.small_scene(seed=seed, n3=50, n4=200)
    a = {k: np.asarray(v, dtype=np.float64) for k, v in scene.arrays().items()}
    a["log_scale4"][:, 3] = 2.0  # wide in time: p(t) ~ 1 everywhere
    rng = np.random.default_rng(seed + 1)
    blocks = [a["sh4"]] + [rng.normal(0, 0.3, a["sh4"].shape) for _ in range(n_time)]
    return a, blocks, views[0]


def _with(a, sh4):
    b = dict(a)
    b["sh4"] = sh4
    return b


def test_zero_higher_blocks_change_nothing():
    a, blocks, view = _scene(2)
    plain = O.render(a, view)["rgb"]
    z = np.concatenate([blocks[0], np.zeros_like(blocks[0]), np.zeros_like(blocks[0])], 1)
    np.testing.assert_array_equal(O.render(_with(a, z), view)["rgb"], plain)


def test_known_cosines_reduce_to_plain_sh():
    a, blocks, view = _scene(2)
    timed = _with(a, np.concatenate(blocks, 1))
    for t, combo in ((0.0, blocks[0] + blocks[1] + blocks[2]),   # all cosines 1
                     (0.25, blocks[0] - blocks[2]),             # cos(pi/2) = 0, cos(pi) = -1
                     (0.5, blocks[0] - blocks[1] + blocks[2])):  # cos(pi) = -1, cos(2 pi) = 1
        v = dataclasses.replace(view, t=t)
        np.testing.assert_allclose(O.project(timed, v)["rgb"], O.project(_with(a, combo), v)["rgb"],
                                   rtol=0, atol=1e-12)


def test_higher_frequencies_average_out_over_the_period():
    a, blocks, view = _scene(2)
    # no space-time coupling (R of Eq. 4 the identity): the sliced mean, hence the view
    # direction, does not move with t
    a["ql"][:] = [1.0, 0.0, 0.0, 0.0]
    a["qr"][:] = [1.0, 0.0, 0.0, 0.0]
    a["sh4"] = blocks[0].copy()
    a["sh4"][:, 0, :] = 20.0  # large DC: no clamp at 0 anywhere
    timed = _with(a, np.concatenate([a["sh4"], blocks[1], blocks[2]], 1))
    M = 16
    acc = 0.0
    for k in range(M):
        acc = acc + O.project(timed, dataclasses.replace(view, t=k / M))["rgb"]
    ref = O.project(a, dataclasses.replace(view, t=0.0))["rgb"]
    vis = O.project(a, dataclasses.replace(view, t=0.0))["visible"] == 1
    np.testing.assert_allclose((acc / M)[vis], ref[vis], rtol=0, atol=1e-12)


def test_conversion_keeps_the_time_constant_block():
    a, blocks, _ = _scene(1)
    a["log_scale4"][:100, 3] = 2.0
    a["log_scale4"][100:, 3] = -2.0
    moved, add, _ = O.convert(_with(a, np.concatenate(blocks, 1)), 1.0)
    np.testing.assert_array_equal(add["sh3"], blocks[0][moved])
