"""The pipelined host-data stepper gives every step's image, loss and
gradients on the host equal to those of a plain device step (images bit for
bit; gradients and loss to atomic-summation rounding), with several steps in
flight -- each slot replaying its captured graph, or issuing the kernels
eagerly."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2, to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graph", [True, False])
def test_pipelined_steps_match_device_step(graph):
    from paper_2412_20522_gb300.hoststep import HostPipeline
    from paper_2412_20522_gb300.rasterize import PARAM_NAMES, RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(40_000, seed=5, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.3, 4.0, 200, 150, 180.0)]
    tgt = torch.as_tensor(scenes.target_image(150, 200, seed=3)).reshape(-1)
    cfg = RasterConfig(bg=(0.1, 0.2, 0.3))
    p = to_device(g)
    rast = Rasterizer()
    img = rast.forward(p, cams, cfg)
    loss, dimg = rast.l1_loss_grad(img, tgt.cuda())
    ref = rast.backward(dimg)
    torch.cuda.synchronize()
    ref_img = img.cpu()
    ref_loss = float(loss.item())
    ref_grads = {k: v.cpu().numpy() for k, v in ref.items()}

    host = {k: v.cpu().pin_memory() for k, v in p.items()}
    hp = HostPipeline(host, tgt.pin_memory(), cams, cfg, graph=graph)
    slots = [hp.step() for _ in range(5)]
    for b in slots[-2:]:
        h_img, h_loss, h_grads = hp.results(b)
        assert torch.equal(h_img, ref_img)
        assert abs(float(h_loss[0]) - ref_loss) < 1e-5 * abs(ref_loss)
        for k in PARAM_NAMES:
            assert rel_l2(h_grads[k].numpy(), ref_grads[k]) < 1e-5, k
    assert hp.h2d_bytes() == sum(v.numel() * v.element_size() for v in host.values()) + tgt.numel() * 4


@pytest.mark.parametrize("graph", [True, False])
def test_pipelined_steps_draw_successive_masks(graph):
    """With the shared device-side iteration, step k of the pipeline samples
    the mask of iteration i0 + k (Sec. 3.3: a new draw every training step)
    and renders what a plain forward with that iteration renders."""
    from paper_2412_20522_gb300.hoststep import HostPipeline
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(20_000, seed=6, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.3, 4.0, 160, 120, 150.0)]
    tgt = torch.as_tensor(scenes.target_image(120, 160, seed=4)).reshape(-1)
    p = to_device(g)
    host = {k: v.cpu().pin_memory() for k, v in p.items()}
    hp = HostPipeline(host, tgt.pin_memory(), cams, RasterConfig(seed=11, iteration=3),
                      graph=graph, advance_iteration=True)
    images = []
    for k in range(3):
        b = hp.step()
        h_img, _, _ = hp.results(b)
        img = Rasterizer().forward(p, cams, RasterConfig(seed=11, iteration=3 + k))
        torch.cuda.synchronize()
        assert torch.equal(h_img, img.cpu()), k
        images.append(h_img.clone())
    assert int(hp.iteration.item()) == 3
    assert not torch.equal(images[0], images[1]) and not torch.equal(images[1], images[2])
