"""The render kernel's fused L1 loss (mg_render_l1) against the separate
render and loss passes: the same image, final T, stop indices and
dL/dimage bit for bit, the loss to rounding (another summation order), on
views of different sizes (per-view normalisation)."""
import math

import pytest
import torch

from gpu_helpers import to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_fused_l1_equals_separate_passes():
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(40_000, seed=51, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(2 * math.pi * k / 3, 4.0, 97 + 31 * k, 61 + 17 * k, 90.0)
            for k in range(3)]
    tgt = torch.cat([torch.as_tensor(scenes.target_image(c.height, c.width, seed=60 + k))
                     .reshape(-1) for k, c in enumerate(cams)]).cuda()
    p = to_device(g)
    cfg = RasterConfig(bg=(0.1, 0.2, 0.3))
    ra, rb = Rasterizer(), Rasterizer()
    img_a = ra.forward(p, cams, cfg).clone()
    loss_a, dimg_a = ra.l1_loss_grad(img_a, tgt)
    loss_a, dimg_a = loss_a.clone(), dimg_a.clone()
    img_b, loss_b, dimg_b = rb.forward_l1(p, cams, cfg, tgt)
    torch.cuda.synchronize()
    assert torch.equal(img_a, img_b)
    for k in ("final_T", "n_contrib"):
        assert torch.equal(ra.splat_outputs()[k], rb.splat_outputs()[k]), k
    assert torch.equal(dimg_a, dimg_b)
    assert abs(float(loss_a) - float(loss_b)) <= 1e-6 * abs(float(loss_a))
    # and the backward from either is the same
    ga = {k: v.clone() for k, v in ra.backward(dimg_a).items()}
    gb = rb.backward(dimg_b)
    torch.cuda.synchronize()
    for k in ga:
        scale = float(ga[k].abs().max()) + 1e-30
        assert float((ga[k] - gb[k]).abs().max()) / scale < 1e-5, k


def test_reset_in_the_render_then_accumulating_backward():
    """mg_render_l1_reset2d zeroes exactly the R rows of grad2d while it
    renders (here filled with NaN first, and a sentinel past them), and
    mg_render_backward_accumulate adding into them gives the 2D gradients of
    mg_render_l1 + mg_render_backward (which resets the rows itself), to
    float-atomic rounding."""
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(30_000, seed=52, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.7, 4.0, 150, 110, 120.0),
            scenes.ring_camera(2.1, 4.0, 90, 70, 80.0)]
    tgt = torch.cat([torch.as_tensor(scenes.target_image(c.height, c.width, seed=70 + k))
                     .reshape(-1) for k, c in enumerate(cams)]).cuda()
    p = to_device(g)
    rast = Rasterizer()
    img, _, dimg = rast.forward_l1(p, cams, RasterConfig(), tgt)
    torch.cuda.synchronize()
    s = rast._state
    R = s["R"]
    F = abi.MG_GRAD2D_FLOATS
    stream = rast._stream()
    buf = rast._buf
    outs = []
    for fused in (False, True):
        g2d = torch.full((R * F + 64,), float("nan"), device="cuda")
        g2d[R * F:] = 7.0                                   # past the rows: untouched
        image = torch.empty_like(img)
        dl = torch.empty_like(dimg)
        loss = torch.zeros(1, device="cuda")
        if fused:
            abi.mg_render_l1_reset2d(s["splats"], s["sorted_vals"], s["ranges"], s["tile_order"],
                                     s["views"], s["V"], s["cfg"], image, buf["final_T"],
                                     buf["n_contrib"], tgt, dl, loss, g2d, stream)
            backward = abi.mg_render_backward_accumulate
        else:
            abi.mg_render_l1(s["splats"], s["sorted_vals"], s["ranges"], s["tile_order"],
                             s["views"], s["V"], s["cfg"], image, buf["final_T"],
                             buf["n_contrib"], tgt, dl, loss, stream)
            backward = abi.mg_render_backward
        backward(s["splats"], s["sorted_vals"], s["ranges"], s["tile_order"], s["views"], s["V"],
                 s["cfg"], buf["final_T"], buf["n_contrib"], dl, g2d, None, stream)
        torch.cuda.synchronize()
        assert torch.equal(image, img) and torch.equal(dl, dimg)
        assert bool(torch.isfinite(g2d[:R * F]).all())
        assert bool((g2d[R * F:] == 7.0).all())
        outs.append(g2d[:R * F].clone())
    scale = float(outs[0].abs().max()) + 1e-30
    assert float((outs[0] - outs[1]).abs().max()) / scale < 1e-5
