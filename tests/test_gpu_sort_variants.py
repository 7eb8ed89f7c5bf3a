"""The autotuner's launch choices that are not tile shapes, each against the
oracle and against the default.

Tile lists, two ways (Sec. 3.1: every tile's Gaussians in depth order, ties
by index):

* "radix8": the records in depth order (4 8-bit passes), the instances
  emitted in that order, then a stable sort by tile id in 8-bit digits;
* "bucket": the instances in record order, grouped by tile in one counting
  pass over the whole tile id, each tile's list then sorted by (depth,
  record) in shared memory -- chunks of 4096 merged for longer lists.

Both must give the same lists bit for bit, hence the same images, final T and
stop indices; the bucket form also passes the full oracle parity check.

Staging depths of the render kernels (splats per shared-memory batch: 256 or
128 in the forward, 128 or 64 in the backward): the per-pixel operation
sequence does not depend on them, so images are bit-identical and gradients
equal to float-atomic rounding; the smaller depths pass the oracle parity.
"""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def _lists(g, cams, cfg_kw=None, capacity=0):
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    out = {}
    dev = to_device(g)
    for mode in ("radix8", "bucket"):
        rast = Rasterizer(capacity=capacity)
        img = rast.forward(dev, cams, RasterConfig(sort=mode, **(cfg_kw or {})))
        torch.cuda.synchronize()
        so = rast.splat_outputs()
        Ks = int(so["num_sorted"].item())
        out[mode] = dict(K=int(so["num_instances"].item()), Ks=Ks,
                         vals=so["sorted_vals"][:Ks].cpu().numpy().copy(),
                         keys=rast.sorted_keys()[:Ks].cpu().numpy().copy(),
                         ranges=so["ranges"].cpu().numpy().reshape(-1, 2).copy(),
                         image=img.clone(), final_T=so["final_T"].clone(),
                         n_contrib=so["n_contrib"].clone())
    return out


def _same(out):
    a, b = out["radix8"], out["bucket"]
    assert a["K"] == b["K"] and a["Ks"] == b["Ks"]
    assert np.array_equal(a["keys"], b["keys"])
    assert np.array_equal(a["vals"], b["vals"])
    ne = a["ranges"][:, 1] > a["ranges"][:, 0]
    assert np.array_equal(a["ranges"][ne], b["ranges"][ne])
    assert (b["ranges"][~ne, 1] == b["ranges"][~ne, 0]).all()
    assert torch.equal(a["image"], b["image"])
    assert torch.equal(a["final_T"], b["final_T"])
    assert torch.equal(a["n_contrib"], b["n_contrib"])


def test_bucket_and_radix_lists_agree_tiny():
    g, cams, _ = scenes.tiny_workload()
    _same(_lists(g, cams))


def test_bucket_and_radix_lists_agree_clusters_multi_view():
    g = scenes.cluster_gaussians(150_000, seed=31)
    cams = [scenes.ring_camera(2 * math.pi * k / 3, 4.0, 500 + 37 * k, 300 + 21 * k, 380.0)
            for k in range(3)]
    _same(_lists(g, cams))
    _same(_lists(g, cams, dict(bin_mode=1, tile_w=32, tile_h=8)))


def test_bucket_merges_lists_longer_than_shared_memory():
    """20 000 small Gaussians crowded into one tile: its list (with ties in
    depth among exact copies) is sorted in 4096-record chunks and merged."""
    g = scenes.uniform_gaussians(24_000, seed=77)
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 128, 96, 110.0)
    Rm = cam.viewmat[:, :3].astype(np.float64)
    tv = cam.viewmat[:, 3].astype(np.float64)
    rng = np.random.default_rng(5)
    m = 20_000
    u = 64.0 + rng.uniform(1.0, 15.0, m)            # inside tile (4, 3) of 16x16 tiles
    v = 48.0 + rng.uniform(1.0, 15.0, m)
    z = 2.0 + rng.uniform(0.0, 2.0, m)
    z[: m // 4] = 2.5                                # exact depth ties
    t = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], 1)
    g.means[:m] = ((t - tv) @ Rm).astype(np.float32)
    g.log_scales[:m] = np.float32(np.log(0.001))
    out = _lists(g, [cam])
    longest = int((out["bucket"]["ranges"][:, 1] - out["bucket"]["ranges"][:, 0]).max())
    assert longest > 4 * 4096
    _same(out)


def test_bucket_parity_with_oracle():
    from test_gpu_parity import _full_check
    from paper_2412_20522_gb300 import rasterize as rz
    g, cams, tgt = scenes.tiny_workload()
    _full_check(rz, g, cams, [tgt], dict(sort="bucket", bg=(0.2, 0.1, 0.4)))
    g = scenes.cluster_gaussians(100_000, seed=8)
    cams = [scenes.ring_camera(0.0, 4.0, 389, 259, 287.5)]
    _full_check(rz, g, cams, [scenes.target_image(259, 389, seed=2)], dict(sort="bucket"))


def test_bucket_capacity_overflow_then_retry():
    """Too small an instance buffer: MG_ERR_CAPACITY with the count needed,
    every range empty; the checked forward grows the buffers and retries."""
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, _ = scenes.tiny_workload()
    dev = to_device(g)
    rast = Rasterizer(capacity=2048)
    img = rast.forward(dev, cams, RasterConfig(sort="bucket"), check=False)
    st = abi.mg_read_status(rast.status, rast._stream())
    assert st.status == abi.MG_ERR_CAPACITY and st.required > 2048
    r = rast.splat_outputs()["ranges"].cpu().numpy().reshape(-1, 2)
    assert (r[:, 1] == r[:, 0]).all()
    ref = _lists(g, cams)["radix8"]
    rast2 = Rasterizer(capacity=2048)
    img = rast2.forward(dev, cams, RasterConfig(sort="bucket"), check=True)
    torch.cuda.synchronize()
    assert torch.equal(img, ref["image"])


def test_bucket_empty_and_culled_scenes():
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.uniform_gaussians(500, seed=1)
    g.means[:, 2] = -10.0
    cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 48, 48, 40.0)]
    rast = Rasterizer()
    img = rast.forward(to_device(g), cams, RasterConfig(sort="bucket", bg=(0.5, 0.5, 0.5)))
    torch.cuda.synchronize()
    assert int(rast.num_sorted.item()) == 0
    assert torch.all(img == 0.5)
    r = rast.splat_outputs()["ranges"].cpu().numpy().reshape(-1, 2)
    assert (r[:, 1] == r[:, 0]).all()


def test_staging_depths_at_parity():
    from test_gpu_parity import _full_check
    from paper_2412_20522_gb300 import rasterize as rz
    kw = dict(render_batch=128, render_batch_bwd=64)
    g, cams, tgt = scenes.tiny_workload()
    _full_check(rz, g, cams, [tgt], dict(kw, bg=(0.3, 0.1, 0.2)))
    g = scenes.cluster_gaussians(100_000, seed=8)
    cams = [scenes.ring_camera(0.0, 4.0, 389, 259, 287.5)]
    _full_check(rz, g, cams, [scenes.target_image(259, 389, seed=2)], dict(kw, sort="bucket"))


def test_staging_depths_change_no_result():
    from gpu_helpers import rel_l2
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(60_000, seed=9)
    cams = [scenes.ring_camera(1.0, 4.0, 300, 200, 230.0)]
    tgt = torch.as_tensor(scenes.target_image(200, 300, seed=3)).cuda().reshape(-1)
    dev = to_device(g)
    res = []
    for fb, bb in ((256, 128), (128, 64), (128, 128), (256, 64)):
        rast = Rasterizer()
        img = rast.forward(dev, cams, RasterConfig(render_batch=fb, render_batch_bwd=bb))
        _, dimg = rast.l1_loss_grad(img, tgt)
        grads = rast.backward(dimg)
        torch.cuda.synchronize()
        res.append((img.clone(), rast.splat_outputs()["n_contrib"].clone(),
                    {k: v.cpu().numpy() for k, v in grads.items()}))
    for img, nc, gr in res[1:]:
        assert torch.equal(img, res[0][0]) and torch.equal(nc, res[0][1])
        for k, v in gr.items():
            assert rel_l2(v, res[0][2][k]) <= 1e-4, k


def test_unsupported_staging_depth_is_rejected():
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, _ = scenes.tiny_workload(500)
    with pytest.raises(abi.MaskgsError) as e:
        Rasterizer().forward(to_device(g), cams, RasterConfig(render_batch=96))
    assert e.value.status == abi.MG_ERR_INVALID_ARG
