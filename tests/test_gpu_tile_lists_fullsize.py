"""The GPU's tile lists at the benchmark's full size (1.2M clustered
Gaussians, 1557x1038, 16x16 tiles), pinned to the paper's definition of which
Gaussians take part in a tile (Sec. 3.1: those intersecting it, with alpha
above zero -- the 3DGS rasteriser's 3-sigma square and 1/255 floor), not to a
restatement of the kernels' own binning optimisation.

* Whole 3-sigma rectangles (MG_BIN_RECT): every Gaussian's tile count, the
  depth order, the instance count, the sorted (tile, record) lists and the
  tile ranges equal, bit for bit, the oracle's plain rectangle emission
  sorted by (tile, depth, index).
* Default (tile-filtered) lists, checked against those rectangle lists with
  nothing of the filter's own code: each tile's list is the rectangle list
  with some pairs removed, order kept; every removed pair has, in FP64 from
  the oracle's splat, a quadratic form above 2 ln 255 at every pixel centre of
  the tile (so alpha < 1/255 for any opacity: the pair is a no-op); and the
  image and final transmittance equal the rectangle run's bit for bit, the
  gradients to atomic-summation rounding.
"""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import PARAMS, rel_l2, to_device
from oracle import binning, fp32_path, pipeline, preprocess
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu

TILE = 16
Q_FLOOR = 2.0 * math.log(255.0)     # alpha = o exp(-q / 2) < 1/255 for o <= 1 beyond it


@pytest.fixture(scope="module")
def runs():
    from paper_2412_20522_gb300.abi import MG_BIN_RECT
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, tgt = scenes.scene_workload()
    dev = to_device(g)
    t = torch.as_tensor(tgt).cuda().reshape(-1)
    out = {}
    for name, cfg in (("rect", RasterConfig(bin_mode=MG_BIN_RECT)), ("filtered", RasterConfig())):
        rast = Rasterizer()
        img = rast.forward(dev, cams, cfg)
        loss, dimg = rast.l1_loss_grad(img, t)
        grads = rast.backward(dimg)
        torch.cuda.synchronize()
        so = rast.splat_outputs()
        K = int(so["num_sorted"].item())
        out[name] = dict(
            image=img.clone(), final_T=so["final_T"].clone(), grads={k: v.clone() for k, v in grads.items()},
            tiles=so["tiles"].cpu().numpy().view(np.uint32).copy(),
            order=(so["order"].cpu().numpy().view(np.uint32).copy()
                   if so["order"] is not None else None),
            K=int(so["num_instances"].item()), Ks=K,
            keys=rast.sorted_keys()[:K].cpu().numpy().view(np.uint32).copy(),
            vals=so["sorted_vals"][:K].cpu().numpy().view(np.uint32).copy(),
            ranges=so["ranges"].cpu().numpy().view(np.uint32).reshape(-1, 2).copy())
        del rast
    return g, cams[0], out


def test_rect_lists_equal_plain_3sigma_emission(runs):
    g, cam, out = runs
    r = out["rect"]
    fp = fp32_path.project32(g.means, g.log_scales, g.quats, cam, TILE, TILE)
    gx, gy = fp["grid"]
    assert np.array_equal(r["tiles"], fp["tiles"])
    if r["order"] is not None:
        assert np.array_equal(r["order"], binning.depth_order(fp["depth_bits"], fp["tiles"] > 0))
    keys, vals, _, K, _ = binning.emit_instances(fp, gx, TILE, TILE)   # every pair kept
    assert r["K"] == K and r["Ks"] == K
    skeys, svals = binning.sort_instances(keys, vals)
    assert np.array_equal(r["keys"].astype(np.uint64), skeys >> np.uint64(32))
    assert np.array_equal(r["vals"], svals)
    ranges = binning.tile_ranges(skeys, gx * gy)
    ne = ranges[:, 1] > ranges[:, 0]
    assert np.array_equal(r["ranges"][ne], ranges[ne])
    assert (r["ranges"][~ne, 0] == r["ranges"][~ne, 1]).all()


def _min_q_over_tile_centres(mean2d, conic, tx, ty, chunk=1 << 16):
    """min over the tile's 16x16 pixel centres of q = d^T Sigma_bar^-1 d, FP64."""
    off = torch.arange(TILE, dtype=torch.float64) + 0.5
    out = np.empty(tx.shape[0])
    for s in range(0, tx.shape[0], chunk):
        e = slice(s, s + chunk)
        m = torch.as_tensor(mean2d[e])
        A, B, C = (torch.as_tensor(conic[e, k])[:, None, None] for k in range(3))
        dx = (torch.as_tensor(tx[e] * TILE, dtype=torch.float64)[:, None] + off) - m[:, 0:1]
        dy = (torch.as_tensor(ty[e] * TILE, dtype=torch.float64)[:, None] + off) - m[:, 1:2]
        q = A * (dx * dx)[:, :, None] + 2.0 * B * dx[:, :, None] * dy[:, None, :] + \
            C * (dy * dy)[:, None, :]
        out[e] = q.reshape(q.shape[0], -1).min(1).values.numpy()
    return out


def test_filtered_lists_are_rect_lists_minus_no_op_pairs(runs):
    g, cam, out = runs
    r, f = out["rect"], out["filtered"]
    R = np.int64(g.n)
    cr = r["keys"].astype(np.int64) * R + r["vals"].astype(np.int64)
    cf = f["keys"].astype(np.int64) * R + f["vals"].astype(np.int64)
    # each kept pair sits in the rectangle lists, in the same order
    srt = np.argsort(cr, kind="stable")
    at = np.searchsorted(cr[srt], cf)
    assert (at < cr.size).all()
    pos = srt[at]
    assert np.array_equal(cr[pos], cf), "a kept pair is not in the rectangle lists"
    assert (np.diff(pos) > 0).all(), "the kept lists do not keep the rectangle order"
    # every removed pair is under the alpha floor at every pixel centre (FP64)
    removed = np.ones(cr.size, bool)
    removed[pos] = False
    rt = r["keys"][removed].astype(np.int64)
    rr = r["vals"][removed].astype(np.int64)
    gx = (cam.width + TILE - 1) // TILE
    vis = np.unique(rr)
    p64 = pipeline.gaussian_params64(g)
    with torch.no_grad():
        sp = preprocess.splat({k: v[torch.as_tensor(vis)] for k, v in p64.items()}, cam)
    idx = np.searchsorted(vis, rr)
    qmin = _min_q_over_tile_centres(sp["mean2d"].numpy()[idx], sp["conic"].numpy()[idx],
                                    rt % gx, rt // gx)
    print(f"rect pairs {cr.size}, kept {cf.size}, removed {rt.size}, "
          f"least removed q {qmin.min() if qmin.size else float('nan'):.4f} (floor {Q_FLOOR:.4f})")
    assert rt.size > 0
    assert (qmin > Q_FLOOR).all(), f"{int((qmin <= Q_FLOOR).sum())} removed pairs reach the floor"


def test_filtered_run_blends_like_rect_run(runs):
    _, _, out = runs
    r, f = out["rect"], out["filtered"]
    assert torch.equal(r["image"], f["image"])
    assert torch.equal(r["final_T"], f["final_T"])
    # gradients: the same terms, summed by float atomics in another order
    # (magnified for thin splats by the chain to their scales and rotations)
    for k in PARAMS:
        e = rel_l2(f["grads"][k].cpu().numpy(), r["grads"][k].cpu().numpy())
        assert e <= 1e-4, (k, e)
