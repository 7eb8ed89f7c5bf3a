"""The longest-first tile order: a permutation of the tile ids whose list
lengths never increase across quarter-octave classes, and a launch order
only -- images and gradients equal those of the tile-id order."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2, to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def _bucket(c):
    c = np.asarray(c, np.int64)
    out = c.copy()
    big = c >= 4
    msb = np.floor(np.log2(np.maximum(c, 1))).astype(np.int64)
    out[big] = 4 * (msb[big] - 1) + ((c[big] >> (msb[big] - 2)) & 3)
    return out


def test_tile_order_is_longest_first_permutation():
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(60_000, seed=31, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.4, 4.0, 333, 250, 300.0),
            scenes.ring_camera(1.4, 4.0, 128, 96, 110.0)]
    rast = Rasterizer()
    rast.forward(to_device(g), cams, RasterConfig())
    torch.cuda.synchronize()
    s = rast._state
    order = s["tile_order"][:s["tiles"]].cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(s["tiles"]))
    rng = s["ranges"][:2 * s["tiles"]].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    b = _bucket(rng[order, 1] - rng[order, 0])
    assert (np.diff(b) <= 0).all()


def test_tile_order_changes_no_result():
    from paper_2412_20522_gb300.rasterize import PARAM_NAMES, RasterConfig, Rasterizer
    g, cams, tgt = scenes.tiny_workload(8000)
    p = to_device(g)
    t = torch.as_tensor(tgt).cuda().reshape(-1)
    outs = []
    for flag in (False, True):
        rast = Rasterizer(tile_order=flag)
        img = rast.forward(p, cams, RasterConfig(bg=(0.3, 0.2, 0.1))).clone()
        _, dimg = rast.l1_loss_grad(img, t)
        grads = {k: v.clone() for k, v in rast.backward(dimg).items()}
        outs.append((img, rast.splat_outputs()["n_contrib"].clone(), grads))
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
    for k in PARAM_NAMES:
        assert rel_l2(outs[1][2][k].cpu().numpy(), outs[0][2][k].cpu().numpy()) < 1e-5, k
