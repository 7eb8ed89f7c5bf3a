"""The depth order is the same whether the preprocess writes the depth keys
(the default) or mg_depth_order derives them from the records, and it is a
permutation with every record that touches no tile last."""
import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from paper_2412_20522_gb300 import abi, scenes

pytestmark = pytest.mark.gpu


def test_depth_order_from_given_or_derived_keys():
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(60_000, seed=33, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.4, 4.0, 333, 250, 300.0),
            scenes.ring_camera(2.0, 4.0, 160, 120, 140.0)]
    rast = Rasterizer()
    rast.forward(to_device(g), cams, RasterConfig())
    s = rast._state
    given = rast.splat_outputs()["order"].clone()
    R = s["R"]
    splats = abi.mg_splats.from_buffer_copy(s["splats"])
    splats.depth_key = None
    dev = given.device
    order, order_alt, keys, keys_alt = (torch.empty(R, dtype=torch.int32, device=dev)
                                        for _ in range(4))
    ws = torch.empty(abi.mg_depth_order_workspace_bytes(R), dtype=torch.uint8, device=dev)
    abi.mg_depth_order(splats, s["views"], s["V"], s["cfg"], order, order_alt, keys, keys_alt,
                       ws, ws.numel(), rast.status, rast._stream())
    torch.cuda.synchronize()
    assert abi.mg_read_status(rast.status, rast._stream()).status == abi.MG_OK
    assert torch.equal(order, given)
    o = order.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(np.sort(o), np.arange(R))
    tiles = rast.splat_outputs()["tiles"].cpu().numpy()
    n_vis = int((tiles > 0).sum())
    assert n_vis > 1000
    assert (tiles[o[:n_vis]] > 0).all() and (tiles[o[n_vis:]] == 0).all()
