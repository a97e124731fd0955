"""The 4D colour with time frequencies (4D spherindrical harmonics) through the
C ABI against the oracle: projection colours, images and every parameter
gradient for views at different timestamps, FP32 and BF16 storage; and the
training kernels that see the wider 4D colour rows (Adam, conversion,
densification)."""
import ctypes as C
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2505_13215_gb300 import abi, raster, scenes, train

from test_gpu_parity import check_grads, check_image, check_projection, loss_grad, make

pytestmark = pytest.mark.gpu


def timed_scene(seed, n_time, n3=2000, n4=2000):
    scene, views = scenes.small_scene(seed=seed, n3=n3, n4=n4)
    rng = np.random.default_rng(seed + 50)
    extra = rng.normal(0, 0.3, (n4, 16 * n_time, 3)).astype(np.float32)
    a = scene.arrays()
    a["sh4"] = np.ascontiguousarray(np.concatenate([a["sh4"], extra], 1))
    return scenes.Scene(**a), views


@pytest.mark.parametrize("dtype,n_time", [(torch.float32, 1), (torch.float32, 3), (torch.bfloat16, 2)])
def test_time_colour_views_match_oracle(dtype, n_time):
    scene, base = timed_scene(60 + n_time, n_time)
    views = [dataclasses.replace(base[0], t=t) for t in (0.13, 0.47, 0.81)]
    G, R = make(scene, views, dtype=dtype)
    assert G.sh_time == n_time
    ref_scene = G.dequantised() if dtype != torch.float32 else scene
    Ps = [O.project(ref_scene, v) for v in views]
    refs = [O.render(ref_scene, v) for v in views]
    for v in range(3):
        check_projection(R, Ps[v], v)
        check_image(R, Ps[v], refs[v], views[v], v)
    dls = loss_grad(R, refs, Ps, views, seed=9)
    check_grads(R, G, ref_scene, Ps, views, dls)


def test_adam_uses_the_dc_step_only_for_the_time_constant_dc():
    scene, _ = timed_scene(70, 2, n3=100, n4=300)
    master = raster.Gaussians.from_scene(scene, "cuda", dtype=torch.float32, capacity3=400)
    s3, s4 = train.AdamState(master, raster.FIELDS3), train.AdamState(master, raster.FIELDS4)
    grads = {k: torch.ones_like(master.t[k][: (master.n3 if k in raster.FIELDS3 else master.n4)])
             for k in raster.FIELDS3 + raster.FIELDS4}
    cg3 = abi.splat_grads3(*[grads[k].data_ptr() for k in raster.FIELDS3])
    cg4 = abi.splat_grads4(*[grads[k].data_ptr() for k in raster.FIELDS4])
    h = abi.splat_adam_hyper()
    for i in range(5):
        h.lr3[i] = 0.0
    for i in range(6):
        h.lr4[i] = 0.0
    h.lr4[5], h.lr_sh_rest, h.beta1, h.beta2, h.eps, h.step = 1e-2, 1e-3, 0.9, 0.999, 1e-30, 1
    before = master.t["sh4"].clone()
    g3, g4 = master.c_g3(), master.c_g4()
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = abi.splat_adam_step(C.byref(h), C.byref(s3.c), C.byref(cg3), C.byref(g3), C.byref(s4.c), C.byref(cg4),
                             C.byref(g4), C.c_void_p(status.data_ptr()),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    step = (before - master.t["sh4"]).cpu().numpy()  # first step with g = 1: the step size itself
    want = np.full(step.shape, 1e-3, dtype=np.float32)
    want[:, 0, :] = 1e-2  # degree 0 of the time-constant block only
    np.testing.assert_allclose(step, want, rtol=0, atol=2e-7)  # FP32 rounding of p - step


def test_conversion_and_densification_carry_the_time_blocks():
    scene, _ = timed_scene(71, 2, n3=300, n4=600)
    a = scene.arrays()
    a["log_scale4"][:300, 3] = 1.0   # static
    a["log_scale4"][300:, 3] = -2.0  # dynamic
    scene = scenes.Scene(**a)
    moved, add, kept = O.convert(scene, 1.0)
    G = raster.Gaussians.from_scene(scene, "cuda", dtype=torch.float32, capacity3=900)
    sh4 = G.t["sh4"].clone()
    m = raster.convert_4d_to_3d(G, 1.0)
    assert m == int(moved.sum())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(G.t["sh3"][300:300 + m].cpu().numpy(), add["sh3"].astype(np.float32))
    assert torch.equal(G.t["sh4"][: G.n4], sh4[torch.from_numpy(kept).cuda()])
    # densification: every 4D Gaussian cloned, full rows copied
    tr_state = raster.Gaussians.from_scene(scene, "cuda", dtype=torch.float32, capacity3=300, capacity4=1200)
    s3, s4 = train.AdamState(tr_state, raster.FIELDS3), train.AdamState(tr_state, raster.FIELDS4)
    n3, n4 = tr_state.n3, tr_state.n4
    tr_state.t["opacity4"][:n4] = 2.0
    tr_state.t["log_scale4"][:n4, :3] = np.log(0.01)
    acc3, cnt3 = torch.zeros(n3, device="cuda"), torch.zeros(n3, device="cuda")
    acc4, cnt4 = torch.ones(n4, device="cuda"), torch.ones(n4, device="cuda")
    nz3, nz4 = torch.zeros(n3, 2, 3, device="cuda"), torch.zeros(n4, 2, 4, device="cuda")
    d3 = abi.splat_densify_set(n3, 300, C.pointer(s3.c), acc3.data_ptr(), cnt3.data_ptr(), nz3.data_ptr(), 0)
    d4 = abi.splat_densify_set(n4, 1200, C.pointer(s4.c), acc4.data_ptr(), cnt4.data_ptr(), nz4.data_ptr(), 2)
    rule = abi.splat_densify_rule(2e-4, 0.05, 5e-3, float(np.log(1.6)))
    wb = abi.splat_densify_workspace_size(n3, 300, n4, 1200, 2)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(2, dtype=torch.int64, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    before = tr_state.t["sh4"][:n4].clone()
    rc = abi.splat_densify(C.byref(rule), C.byref(d3), C.byref(d4), C.c_void_p(n_out.data_ptr()),
                           C.c_void_p(status.data_ptr()), C.c_void_p(ws.data_ptr()), wb,
                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == abi.SPLAT_OK
    torch.cuda.synchronize()
    assert int(status[0]) == 0 and int(n_out[1]) == 2 * n4
    assert torch.equal(tr_state.t["sh4"][:n4], before) and torch.equal(tr_state.t["sh4"][n4:2 * n4], before)
