"""A step captured in a CUDA graph keeps the arguments it was captured with,
the mask sample's iteration among them.  With the iteration in a device
counter that the step advances (mg_raster_cfg.iteration_dev,
mg_advance_iteration), successive replays draw successive Gumbel masks
(Sec. 3.3): replay k samples with iteration i0 + k, bit-equal to the oracle's
mask for that iteration, and renders the image a plain forward with that
iteration renders."""
import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from oracle import fp32_path
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_replays_draw_successive_masks():
    from paper_2412_20522_gb300.autotune import GraphStep
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, tgt = scenes.tiny_workload(8000)
    p = to_device(g)
    target = torch.as_tensor(tgt).reshape(-1).cuda()
    cfg = RasterConfig(seed=77, iteration=5)
    gs = GraphStep(p, cams, cfg, target, advance_iteration=True)
    gs.iteration.fill_(0)                 # the next replay samples with iteration 5
    masks = []
    for k in range(3):
        gs.replay()
        torch.cuda.synchronize()
        assert gs.status() == 0
        assert int(gs.iteration.item()) == k + 1
        m = gs.rast.splat_outputs()["mask"].cpu().numpy().astype(bool)
        ref = fp32_path.sample_mask(g.mask_logits, 77, 5 + k)[0].astype(bool)
        assert np.array_equal(m, ref), k
        masks.append(m)
        # the image a plain forward with that iteration renders
        rast = Rasterizer()
        img = rast.forward(p, cams, RasterConfig(seed=77, iteration=5 + k))
        torch.cuda.synchronize()
        assert torch.equal(img, gs.image), k
    assert not np.array_equal(masks[0], masks[1]) and not np.array_equal(masks[1], masks[2])
