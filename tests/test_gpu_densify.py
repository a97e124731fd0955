"""Densification through the C ABI against the oracle: the statistics of the
projected-mean gradients, and the clone / split / prune pass on both sets
(including the optimizer state and the capacity check)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_13215_gb300 import abi, raster, scenes, train

from parity_util import assert_split_means


pytestmark = pytest.mark.gpu

F3, F4 = raster.FIELDS3, raster.FIELDS4
RULE = dict(grad_threshold=2e-4, dense_scale=0.05, min_opacity=5e-3, split_shrink=float(np.float32(np.log(1.6))))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_densify_stats_accumulate_ndc_gradient_norms():
    scene, views = scenes.small_scene(seed=40)
    G = raster.Gaussians.from_scene(scene, "cuda")
    R = raster.Rasterizer(G.n3, G.n4, views)
    R.autotune_capacity(G)
    R.forward(G)
    dl = torch.randn(R.rgb.shape, device="cuda") * 1e-3
    R.backward(G, dl, stop_2d=True)
    torch.cuda.synchronize()
    R.check()
    acc = torch.zeros(R.N, device="cuda")
    cnt = torch.zeros(R.N, device="cuda")
    for _ in range(2):
        rc = abi.splat_densify_stats(C.byref(R.cproj), R.cviews, R.V, C.c_void_p(R.dproj.data_ptr()),
                                     C.c_void_p(acc.data_ptr()), C.c_void_p(cnt.data_ptr()), _stream())
        assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    dp = R.dproj.view(-1, 12)[:, :2].double().cpu().numpy()
    vis = R.n_tiles.cpu().numpy() > 0
    want_a, want_c = O.densify_stats(dp, vis, views[0].W, views[0].H)
    np.testing.assert_array_equal(cnt.cpu().numpy(), 2 * want_c)
    np.testing.assert_allclose(acc.double().cpu().numpy(), 2 * want_a, rtol=2e-6, atol=1e-12)


def _random_state(n3, cap3, n4, cap4, seed):
    """FP32 master sets with Adam moments, statistics and draws; no decision within
    0.1% of its threshold, so FP32 and FP64 classify alike."""
    scene, _ = scenes.small_scene(seed=seed, n3=n3, n4=n4)
    rng = np.random.default_rng(seed)
    a = scene.arrays()
    # opacities, statistics and scales spread over both sides of each threshold
    a["opacity3"][:] = rng.choice([-8.0, -6.0, 0.5, 2.0], n3).astype(np.float32)
    a["opacity4"][:] = rng.choice([-8.0, -6.0, 0.5, 2.0], n4).astype(np.float32)
    a["log_scale3"][:] = rng.choice([np.log(0.02), np.log(0.1)], (n3, 1)).astype(np.float32) + \
        rng.normal(0, 0.1, (n3, 3)).astype(np.float32)
    a["log_scale4"][:] = rng.choice([np.log(0.02), np.log(0.1)], (n4, 1)).astype(np.float32) + \
        rng.normal(0, 0.1, (n4, 4)).astype(np.float32)
    for k in ("log_scale3", "log_scale4"):
        mx = np.exp(a[k][:, :3].astype(np.float64).max(1))
        ok = np.abs(mx / RULE["dense_scale"] - 1) > 1e-3
        a[k][~ok] -= np.float32(0.2)
    master = raster.Gaussians.from_scene(scenes.Scene(**a), "cuda", dtype=torch.float32, capacity3=cap3)
    for k in F4:  # 4D rows up to cap4
        pad = torch.zeros((cap4 - n4,) + raster.SHAPES[k], device="cuda")
        master.t[k] = torch.cat([master.t[k], pad], 0).contiguous()
    s3, s4 = train.AdamState(master, F3), train.AdamState(master, F4)
    for s in (s3, s4):
        for k in s.fields:
            s.m[k].normal_()
            s.v[k].uniform_(0.1, 1.0)
    stats = {}
    for name, n in (("3", n3), ("4", n4)):
        cnt = rng.integers(0, 4, n).astype(np.float32)
        avg = rng.choice([5e-5, 1e-4, 3e-4, 9e-4], n)
        stats[name] = (torch.from_numpy((avg * cnt).astype(np.float32)).cuda(), torch.from_numpy(cnt).cuda())
    noise3 = torch.randn((n3, 2, 3), device="cuda")
    noise4 = torch.randn((n4, 2, 4), device="cuda")
    return master, s3, s4, stats, noise3, noise4


def _dset(n, cap, state, stats, noise):
    return abi.splat_densify_set(n, cap, C.pointer(state.c), stats[0].data_ptr(), stats[1].data_ptr(),
                                 noise.data_ptr())


def _rule():
    r = abi.splat_densify_rule()
    r.grad_threshold, r.dense_scale, r.min_opacity, r.split_shrink = (RULE["grad_threshold"], RULE["dense_scale"],
                                                                      RULE["min_opacity"], RULE["split_shrink"])
    return r


def test_densify_matches_oracle_on_both_sets():
    n3, cap3, n4, cap4 = 600, 2000, 500, 1600
    master, s3, s4, stats, noise3, noise4 = _random_state(n3, cap3, n4, cap4, seed=41)
    before = {k: master.t[k][: (n3 if k in F3 else n4)].double().cpu().numpy() for k in F3 + F4}
    m0 = {k: (s3 if k in F3 else s4).m[k][: (n3 if k in F3 else n4)].double().cpu().numpy() for k in F3 + F4}
    v0 = {k: (s3 if k in F3 else s4).v[k][: (n3 if k in F3 else n4)].double().cpu().numpy() for k in F3 + F4}
    wb = abi.splat_densify_workspace_size(n3, cap3, n4, cap4)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(2, dtype=torch.int64, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    d3 = _dset(n3, cap3, s3, stats["3"], noise3)
    d4 = _dset(n4, cap4, s4, stats["4"], noise4)
    rc = abi.splat_densify(C.byref(_rule()), C.byref(d3), C.byref(d4), C.c_void_p(n_out.data_ptr()),
                           C.c_void_p(status.data_ptr()), C.c_void_p(ws.data_ptr()), wb, _stream())
    assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    assert int(status[0]) == 0, abi.status_string(int(status[0]))
    for four_d, fields, (acc, cnt), noise, s in ((False, F3, stats["3"], noise3, s3), (True, F4, stats["4"], noise4, s4)):
        want_p, want_m, want_v = O.densify_set({k: before[k] for k in fields}, {k: m0[k] for k in fields},
                                               {k: v0[k] for k in fields}, acc.double().cpu().numpy(),
                                               cnt.double().cpu().numpy(), noise.double().cpu().numpy(),
                                               four_d=four_d, **RULE)
        n_new = int(n_out[1 if four_d else 0])
        assert n_new == want_p[fields[0]].shape[0]
        assert n_new != (n4 if four_d else n3)  # something happened
        for k in fields:
            got = master.t[k][:n_new].double().cpu().numpy()
            if k in ("mean3", "mean4"):  # FP32 sums of O(1) offsets: the derived bound
                assert_split_means(got, want_p[k], want_p["log_scale4" if four_d else "log_scale3"],
                                   noise.double().cpu().numpy(), RULE["split_shrink"], k)
            elif k in ("log_scale3", "log_scale4"):
                np.testing.assert_allclose(got, want_p[k], rtol=0, atol=1e-6, err_msg=k)
            else:
                np.testing.assert_array_equal(got, want_p[k], err_msg=k)
            np.testing.assert_array_equal(s.m[k][:n_new].double().cpu().numpy(), want_m[k], err_msg=k)
            np.testing.assert_array_equal(s.v[k][:n_new].double().cpu().numpy(), want_v[k], err_msg=k)


def test_densify_capacity_overflow_changes_nothing():
    n3, n4 = 600, 500
    master, s3, s4, stats, noise3, noise4 = _random_state(n3, n3 + 100, n4, n4 + 100, seed=42)
    # every 4D Gaussian densifies and none is pruned: the 4D set outgrows its capacity
    master.t["opacity4"].fill_(2.0)
    stats["4"][0].fill_(1.0)
    stats["4"][1].fill_(1.0)
    before = {k: master.t[k].clone() for k in F3 + F4}
    wb = abi.splat_densify_workspace_size(n3, n3 + 100, n4, n4 + 100)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(2, dtype=torch.int64, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    d3, d4 = _dset(n3, n3 + 100, s3, stats["3"], noise3), _dset(n4, n4 + 100, s4, stats["4"], noise4)
    rc = abi.splat_densify(C.byref(_rule()), C.byref(d3), C.byref(d4), C.c_void_p(n_out.data_ptr()),
                           C.c_void_p(status.data_ptr()), C.c_void_p(ws.data_ptr()), wb, _stream())
    assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    assert int(n_out[1]) > n4 + 100
    assert int(status[0]) == abi.SPLAT_ERR_CAPACITY and int(status[1]) == 10
    for k in F3 + F4:  # neither set changed
        assert torch.equal(master.t[k], before[k]), k
