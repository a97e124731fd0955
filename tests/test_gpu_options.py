"""Per-rasterizer tuning through splat_options, in one process.

Two rasterizers of the same scene run interleaved with different settings --
pixels per lane, tile sort mode (radix passes / binned partition) and
footprint culling with the saturation cut -- while the library-wide defaults
(splat_set_*) point elsewhere.  Each rasterizer must see its own settings
(the lists it builds, the pair counts it records) and both must render the
same image and gradients, which do not depend on the tuning; the library-wide
defaults are left as they were.
"""
import numpy as np
import pytest
import torch

from paper_2505_13215_gb300 import abi, raster, scenes

from parity_util import rel_l2

pytestmark = pytest.mark.gpu


def test_two_rasterizers_with_their_own_options():
    scene, views = scenes.arc_scene(seed=21, n=40000, frac4=0.3, n_views=2, full=(320, 240, 350.0),
                                    half=(200, 150, 220.0))
    G = raster.Gaussians.from_scene(scene, "cuda")
    target = torch.rand(sum(3 * v.W * v.H for v in views), generator=torch.Generator(device="cuda").manual_seed(3),
                        device="cuda")
    Ra = raster.Rasterizer(G.n3, G.n4, views)
    Rb = raster.Rasterizer(G.n3, G.n4, views)
    ca = torch.zeros(8, dtype=torch.int64, device="cuda")
    cb = torch.zeros(8, dtype=torch.int64, device="cuda")
    Ra.set_options(ppl_fwd=2, ppl_bwd=4, tile_sort=1, tile_cull=0, stats=ca.data_ptr())
    Rb.set_options(ppl_fwd=8, ppl_bwd=8, tile_sort=2, tile_cull=1, stats=cb.data_ptr())
    # library-wide defaults that neither rasterizer should follow
    abi.splat_set_pixels_per_lane(4, 4)
    abi.splat_set_tile_cull(False)
    try:
        Ra.autotune_capacity(G)
        Rb.autotune_capacity(G)
        ca.zero_()
        cb.zero_()
        for _ in range(2):  # interleaved steps
            Ra.step(G, target)
            Rb.step(G, target)
        torch.cuda.synchronize()
        Ra.check("a")
        Rb.check("b")
        # unculled lists hold every tile of every rectangle; the culled, cut lists fewer
        assert Ra.instances() == int(Ra.n_tiles.sum().item())
        assert Rb.instances() < Ra.instances()
        assert Ra.keep_keys and bool((Ra.keys[1:Ra.instances()] >= Ra.keys[:Ra.instances() - 1]).all())
        # the pair counters of each rasterizer's own calls (two steps each)
        fa, fb = ca.cpu().numpy(), cb.cpu().numpy()
        assert fa[0] > 0 and fb[0] > 0 and fa[2] > 0 and fb[2] > 0
        # the sort's counters: only the binned, culled path has tail segments to count
        assert fa[4] == 0 and fa[5] == 0
        # the result does not depend on the tuning
        assert torch.equal(Ra.rgb, Rb.rgb) and torch.equal(Ra.final_T, Rb.final_T)
        for k in raster.FIELDS3 + raster.FIELDS4:
            assert rel_l2(Ra.grads[k].cpu().numpy(), Rb.grads[k].cpu().numpy()) < 1e-5, k
        # a third rasterizer left at the library defaults follows them (no culling now)
        Rc = raster.Rasterizer(G.n3, G.n4, views)
        Rc.autotune_capacity(G)
        Rc.step(G, target)
        torch.cuda.synchronize()
        Rc.check("c")
        assert Rc.instances() == Ra.instances()
        assert torch.equal(Rc.rgb, Rb.rgb)
    finally:
        abi.splat_set_pixels_per_lane(8, 8)
        abi.splat_set_tile_cull(True)
