"""The training step's own kernels through the C ABI: the fused Adam launch
against the oracle's Adam, the storage cast, the optimizer-state side of the
4D -> 3D conversion against the oracle's conversion, and the Trainer that
chains render, loss, backward, Adam and conversion."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_13215_gb300 import abi, raster, scenes, train

from parity_util import assert_split_means

pytestmark = pytest.mark.gpu

F3, F4 = raster.FIELDS3, raster.FIELDS4
LR3 = {"mean3": 1e-3, "log_scale3": 5e-3, "quat3": 2e-3, "opacity3": 5e-2, "sh3": 3e-3}
LR4 = {"mean4": 7e-4, "log_scale4": 4e-3, "ql": 1e-3, "qr": 1.5e-3, "opacity4": 4e-2, "sh4": 2e-3}
LR_REST = 1.5e-4
# the hyperparameters travel as FP32 numbers: the oracle gets the same values
B1, B2 = float(np.float32(0.9)), float(np.float32(0.999))


def _hyper(step, b1=0.9, b2=0.999, eps=1e-15):
    h = abi.splat_adam_hyper()
    for i, k in enumerate(F3):
        h.lr3[i] = LR3[k]
    for i, k in enumerate(F4):
        h.lr4[i] = LR4[k]
    h.lr_sh_rest, h.beta1, h.beta2, h.eps, h.step = LR_REST, b1, b2, eps, step
    return h


def _lr_array(k, n):
    shape = (n,) + raster.SHAPES[k]
    lr = np.full(shape, (LR3 if k in F3 else LR4)[k])
    if k in ("sh3", "sh4"):
        lr[:, 1:, :] = LR_REST  # degree >= 1
    return lr


def _scene_with_time_scales(seed, n3, n4, tau):
    scene, views = scenes.small_scene(seed=seed, n3=n3, n4=n4)
    rng = np.random.default_rng(seed + 100)
    # half static, half dynamic, none within 5% of the threshold
    st = np.where(rng.uniform(size=n4) < 0.5, rng.uniform(0.1, 1.5, n4), rng.uniform(-3.0, -0.1, n4))
    scene.log_scale4[:, 3] = (st + np.log(tau)).astype(np.float32)
    return scene, views


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_adam_step_matches_oracle(dtype):
    scene, _ = scenes.small_scene(seed=21, n3=700, n4=500)
    cap3 = 1000
    master = raster.Gaussians.from_scene(scene, "cuda", dtype=torch.float32, capacity3=cap3)
    store = master if dtype == torch.float32 else raster.Gaussians.from_scene(scene, "cuda", dtype=dtype,
                                                                               capacity3=cap3)
    s3, s4 = train.AdamState(master, F3), train.AdamState(master, F4)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    want = {k: (master.t[k][: (master.n3 if k in F3 else master.n4)].double().cpu().numpy(), 0.0, 0.0)
            for k in F3 + F4}
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for t in range(1, 4):
        grads = {k: torch.randn((master.n3 if k in F3 else master.n4,) + raster.SHAPES[k], generator=gen,
                                device="cuda") for k in F3 + F4}
        cg3 = abi.splat_grads3(*[grads[k].data_ptr() for k in F3])
        cg4 = abi.splat_grads4(*[grads[k].data_ptr() for k in F4])
        g3, g4 = store.c_g3(), store.c_g4()
        rc = abi.splat_adam_step(C.byref(_hyper(t)), C.byref(s3.c), C.byref(cg3), C.byref(g3), C.byref(s4.c),
                                 C.byref(cg4), C.byref(g4), C.c_void_p(status.data_ptr()), stream)
        assert rc == abi.SPLAT_OK
        for k in F3 + F4:
            p, m, v = want[k]
            g = grads[k].double().cpu().numpy()
            want[k] = O.adam_step(p, m, v, g, t, _lr_array(k, g.shape[0]), B1, B2, 1e-15)
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    for k in F3 + F4:
        n = master.n3 if k in F3 else master.n4
        p, m, v = want[k]
        s = s3 if k in F3 else s4
        np.testing.assert_allclose(s.m[k][:n].double().cpu().numpy(), m, rtol=2e-6, atol=1e-7, err_msg=k)
        np.testing.assert_allclose(s.v[k][:n].double().cpu().numpy(), v, rtol=2e-6, atol=1e-9, err_msg=k)
        lr = max(LR3.get(k, 0.0), LR4.get(k, 0.0))
        np.testing.assert_allclose(master.t[k][:n].double().cpu().numpy(), p, rtol=1e-6, atol=1e-5 * lr, err_msg=k)
        # the storage copy is the master rounded to nearest; rows past n untouched
        assert torch.equal(store.t[k][:n], master.t[k][:n].to(dtype)), k
    if dtype != torch.float32:
        assert torch.count_nonzero(store.t["mean3"][master.n3:]) == 0


def test_cast_params_rounds_to_nearest():
    scene, _ = scenes.small_scene(seed=22, n3=300, n4=200)
    master = raster.Gaussians.from_scene(scene, "cuda", dtype=torch.float32, capacity3=400)
    for k in F3 + F4:
        master.t[k].mul_(1.0 + 1e-3 * torch.rand_like(master.t[k]))
    for dtype in (torch.bfloat16, torch.float16):
        dst = raster.Gaussians.from_scene(scenes.empty_scene(), "cuda", dtype=dtype, capacity3=400)
        dst.t = {k: torch.zeros_like(master.t[k], dtype=dtype) for k in F3 + F4}
        dst.n3, dst.n4 = master.n3, master.n4
        s3, s4, d3, d4 = master.c_g3(), master.c_g4(), dst.c_g3(), dst.c_g4()
        rc = abi.splat_cast_params(C.byref(s3), C.byref(d3), C.byref(s4), C.byref(d4),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == abi.SPLAT_OK
        torch.cuda.synchronize()
        for k in F3 + F4:
            n = master.n3 if k in F3 else master.n4
            assert torch.equal(dst.t[k][:n], master.t[k][:n].to(dtype)), k


def test_convert_adam_state_follows_the_oracle_conversion():
    tau = 1.0
    scene, _ = _scene_with_time_scales(23, 300, 1000, tau)
    moved_mask, _, kept = O.convert(scene, tau)
    moved_mask = moved_mask.astype(bool)
    cap3 = 1500
    master = raster.Gaussians.from_scene(scene, "cuda", dtype=torch.float32, capacity3=cap3)
    s3, s4 = train.AdamState(master, F3), train.AdamState(master, F4)
    for s in (s3, s4):
        for k in s.fields:
            s.m[k].normal_()
            s.v[k].uniform_(0.1, 1.0)
    m3_0 = {k: s3.m[k].clone() for k in F3}
    m4_0 = {k: s4.m[k].clone() for k in F4}
    v4_0 = {k: s4.v[k].clone() for k in F4}
    wb = abi.splat_workspace_size(abi.SPLAT_OP_CONVERT_STATE, 0, master.n4, [16], [16], 0)
    ws = torch.empty(int(wb), dtype=torch.uint8, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    g3, g4 = master.c_g3(), master.c_g4()
    rc = abi.splat_convert_adam_state(C.byref(g4), C.byref(g3), tau, C.byref(s4.c), C.byref(s3.c),
                                      C.c_void_p(status.data_ptr()), C.c_void_p(ws.data_ptr()), wb,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    assert int(status[0]) == 0
    n3, moved = master.n3, int(moved_mask.sum())
    assert 0 < moved < master.n4
    kept_t = torch.from_numpy(np.asarray(kept, dtype=np.int64)).cuda()
    for k in F4:
        assert torch.equal(s4.m[k][: len(kept)], m4_0[k][kept_t]), k
        assert torch.equal(s4.v[k][: len(kept)], v4_0[k][kept_t]), k
    for k in F3:
        assert torch.count_nonzero(s3.m[k][n3:n3 + moved]) == 0, k
        assert torch.count_nonzero(s3.v[k][n3:n3 + moved]) == 0, k
        assert torch.equal(s3.m[k][:n3], m3_0[k][:n3]), k
        assert torch.equal(s3.m[k][n3 + moved:], m3_0[k][n3 + moved:]), k


def test_trainer_step_and_conversion():
    tau = 1.0
    scene, views = _scene_with_time_scales(24, 800, 1200, tau)
    tr = train.Trainer(scene, views, dtype=torch.bfloat16, tau=tau, convert_every=0)
    target_scene, _ = scenes.small_scene(seed=25, n3=800, n4=1200)
    target = torch.from_numpy(O.render(target_scene, views[0])["rgb"].reshape(-1)).float().cuda()
    p0 = {k: tr.master.t[k][: (tr.n3 if k in F3 else tr.n4)].double().cpu().numpy() for k in F3 + F4}
    tr.step(views, target)
    torch.cuda.synchronize()
    tr.R.check("train step")
    loss0 = float(tr.loss.item())
    # one Adam step from zero moments on the step's own gradients
    for k in F3 + F4:
        n = tr.n3 if k in F3 else tr.n4
        g = tr.R.grads[k].double().cpu().numpy()
        p, _, _ = O.adam_step(p0[k], 0.0, 0.0, g, 1, _trainer_lr(tr, k, n), B1, B2, 1e-15)
        np.testing.assert_allclose(tr.master.t[k][:n].double().cpu().numpy(), p, rtol=1e-6, atol=1e-7, err_msg=k)
        assert torch.equal(tr.store.t[k][:n], tr.master.t[k][:n].to(torch.bfloat16)), k
    # conversion: the master sets become the oracle's conversion of the current master
    cur = {k: tr.master.t[k][: (tr.n3 if k in F3 else tr.n4)].double().cpu().numpy() for k in F3 + F4}
    moved_mask, add3, kept = O.convert(cur, tau)
    n3_before = tr.n3
    moved = tr.convert()
    assert moved == int(moved_mask.sum()) > 0
    assert tr.n3 == n3_before + moved and tr.n4 == 1200 - moved
    np.testing.assert_array_equal(tr.master.t["mean4"][: tr.n4].cpu().numpy(), cur["mean4"][kept].astype(np.float32))
    np.testing.assert_array_equal(tr.master.t["mean3"][n3_before: tr.n3].cpu().numpy(),
                                  add3["mean3"].astype(np.float32))
    np.testing.assert_allclose(tr.master.t["quat3"][n3_before: tr.n3].cpu().numpy(), add3["quat3"], atol=2e-5)
    for k in F3 + F4:
        n = tr.n3 if k in F3 else tr.n4
        assert torch.equal(tr.store.t[k][:n], tr.master.t[k][:n].to(torch.bfloat16)), k
    # training goes on with the new split, and the loss goes down
    for _ in range(30):
        tr.step(views, target)
    torch.cuda.synchronize()
    tr.R.check("train steps")
    assert float(tr.loss.item()) < loss0


def _trainer_lr(tr, k, n):
    lr = np.full((n,) + raster.SHAPES[k], tr.hyper.lr3[F3.index(k)] if k in F3 else tr.hyper.lr4[F4.index(k)])
    if k in ("sh3", "sh4"):
        lr[:, 1:, :] = tr.hyper.lr_sh_rest
    return lr


def test_trainer_densification_matches_oracle():
    """Statistics gathered over the steps, then Trainer.densify: both master sets and
    their moments equal the oracle's densification of the snapshot, with the same
    N(0, 1) draws (the CUDA generator reseeded)."""
    scene, views = _scene_with_time_scales(26, 900, 900, 1.0)
    rule = {"grad_threshold": 1e-5, "dense_scale": 0.04}  # low threshold: the few steps densify something
    tr = train.Trainer(scene, views, dtype=torch.bfloat16, convert_every=0, densify_every=1000, densify=rule)
    target = torch.rand(tr.R.rgb.shape, device="cuda")
    for _ in range(4):
        tr.step(views, target)
    torch.cuda.synchronize()
    n3, n4 = tr.n3, tr.n4
    snap = {k: tr.master.t[k][: (n3 if k in F3 else n4)].double().cpu().numpy() for k in F3 + F4}
    mom = {k: ((tr.s3 if k in F3 else tr.s4).m[k][: (n3 if k in F3 else n4)].double().cpu().numpy(),
               (tr.s3 if k in F3 else tr.s4).v[k][: (n3 if k in F3 else n4)].double().cpu().numpy())
           for k in F3 + F4}
    acc = tr.accum.double().cpu().numpy()
    cnt = tr.count.double().cpu().numpy()
    torch.manual_seed(123)
    noise3 = torch.randn((max(1, n3), 2, 3), device="cuda").double().cpu().numpy()
    noise4 = torch.randn((max(1, n4), 2, 4), device="cuda").double().cpu().numpy()
    torch.manual_seed(123)
    new3, new4 = tr.densify()
    full = dict(train.DEFAULT_DENSIFY, **rule)
    full = {k: float(np.float32(v)) for k, v in full.items()}
    for four_d, fields, lo, hi, noise, n_new, s in ((False, F3, n4, n4 + n3, noise3, new3, tr.s3),
                                                    (True, F4, 0, n4, noise4, new4, tr.s4)):
        want_p, want_m, want_v = O.densify_set({k: snap[k] for k in fields}, {k: mom[k][0] for k in fields},
                                               {k: mom[k][1] for k in fields}, acc[lo:hi], cnt[lo:hi], noise,
                                               four_d=four_d, **full)
        assert n_new == want_p[fields[0]].shape[0]
        for k in fields:
            got = tr.master.t[k][:n_new].double().cpu().numpy()
            if k in ("mean3", "mean4"):  # FP32 sums of O(1) offsets: the derived bound
                assert_split_means(got, want_p[k], want_p["log_scale4" if four_d else "log_scale3"], noise,
                                   full["split_shrink"], k)
                continue
            tol = 1e-6 if k in ("log_scale3", "log_scale4") else 0.0
            np.testing.assert_allclose(got, want_p[k], rtol=tol, atol=tol, err_msg=k)
            np.testing.assert_array_equal(s.m[k][:n_new].double().cpu().numpy(), want_m[k], err_msg=k)
            assert torch.equal(tr.store.t[k][:n_new], tr.master.t[k][:n_new].to(torch.bfloat16)), k
    assert (new3, new4) != (n3, n4)
    # training goes on with the new counts
    for _ in range(3):
        tr.step(views, target)
    torch.cuda.synchronize()
    tr.R.check("after densification")
    assert np.isfinite(float(tr.loss.item()))


def test_checkpoint_resume_continues_identically(tmp_path):
    """state_dict after a few steps, a fresh Trainer loaded from it: the same state bit
    for bit; one more step on both: the same parameters up to the order of the
    gradient atomics."""
    scene, views = _scene_with_time_scales(27, 700, 700, 1.0)
    target = torch.rand((3 * 128 * 128,), device="cuda")
    a = train.Trainer(scene, views, dtype=torch.bfloat16, convert_every=2)
    for _ in range(3):  # includes a conversion
        a.step(views, target)
    path = tmp_path / "ckpt.pt"
    torch.save(a.state_dict(), path)
    b = train.Trainer(scene, views, dtype=torch.bfloat16, convert_every=2)
    b.load_state_dict(torch.load(path))
    assert (b.n3, b.n4, b.t) == (a.n3, a.n4, a.t)
    for k in F3 + F4:
        n = a.n3 if k in F3 else a.n4
        assert torch.equal(a.master.t[k][:n], b.master.t[k][:n]), k
        assert torch.equal(a.store.t[k][:n], b.store.t[k][:n]), k
        st_a, st_b = (a.s3, b.s3) if k in F3 else (a.s4, b.s4)
        assert torch.equal(st_a.m[k][:n], st_b.m[k][:n]) and torch.equal(st_a.v[k][:n], st_b.v[k][:n]), k
    for tr in (a, b):
        tr.step(views, target)
    torch.cuda.synchronize()
    for k in F3 + F4:
        n = a.n3 if k in F3 else a.n4
        pa, pb = a.master.t[k][:n].double().cpu().numpy(), b.master.t[k][:n].double().cpu().numpy()
        assert np.abs(pa - pb).max() <= 1e-6 * max(1.0, np.abs(pa).max()), k
