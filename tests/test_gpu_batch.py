"""Batched forms: a CUDA-graph replay of the whole step equals the eager step
bit for bit; an uneven batch of scenes (disjoint Gaussian ranges, one camera
each, mixed resolutions) in one launch sequence matches the oracle per scene;
the tile-shape autotuner picks a measured shape and caches it."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2, to_device
from oracle import pipeline
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_graph_replay_equals_eager_step():
    from paper_2412_20522_gb300.autotune import GraphStep
    from paper_2412_20522_gb300.rasterize import PARAM_NAMES, RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(30_000, seed=3, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(2 * math.pi * k / 4, 4.0, 160, 120, 130.0) for k in range(4)]
    tgt = torch.cat([torch.as_tensor(scenes.target_image(c.height, c.width, seed=k)).reshape(-1)
                     for k, c in enumerate(cams)]).cuda()
    p = to_device(g)
    cfg = RasterConfig(bg=(0.1, 0.2, 0.3), seed=9, iteration=4)
    gs = GraphStep(p, cams, cfg, tgt)
    gs.replay()
    gs.replay()
    torch.cuda.synchronize()
    assert gs.status() == 0
    rast = Rasterizer()
    img = rast.forward(p, cams, cfg)
    loss, dimg = rast.l1_loss_grad(img, tgt)
    grads = rast.backward(dimg)
    torch.cuda.synchronize()
    assert torch.equal(img, gs.image)
    for k in PARAM_NAMES:
        # atomics may reorder FP32 sums: equal up to rounding
        assert rel_l2(gs.grads[k].cpu().numpy(), grads[k].cpu().numpy()) < 1e-5, k
    assert abs(float(loss) - float(gs.loss)) < 1e-5 * abs(float(loss))    # atomic sum


def _tile_lists(rast, t0, nt, r0):
    so = rast.splat_outputs()
    rng = so["ranges"].cpu().numpy().view(np.uint32).reshape(-1, 2)[t0:t0 + nt]
    vals = so["sorted_vals"].cpu().numpy().view(np.uint32)
    return [vals[s:e].astype(np.int64) - r0 for s, e in rng]


@pytest.mark.parametrize("lambda_m", [0.0, 0.3])
def test_uneven_scene_batch_matches_oracle_per_scene(lambda_m):
    """With lambda_m > 0 every scene has its own mask loss L_m over its own
    N Gaussians (Eq. 7), so the mask-logit gradients differ per scene."""
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    sizes = [1500, 4000, 9000]
    sc = [scenes.cluster_gaussians(n, seed=40 + k, centre_radius=1.5, reject_radius=2.0,
                                   log_scale_mu=-4.0, log_scale_sigma=0.5)
          for k, n in enumerate(sizes)]
    cams = [scenes.ring_camera(0.7 * k, 4.0, w, h, 0.8 * w)
            for k, (w, h) in enumerate([(72, 48), (100, 75), (131, 97)])]
    cat = {k: np.concatenate([getattr(s, k) for s in sc]) for k in
           ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")}
    gall = scenes.Gaussians(**cat, sh_degree=3)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    ranges = [(int(o), n) for o, n in zip(offs, sizes)]
    cfg = RasterConfig(bg=(0.3, 0.3, 0.3), seed=77, iteration=2, lambda_m=lambda_m)
    rast = Rasterizer()
    img = rast.forward(to_device(gall), cams, cfg, view_ranges=ranges)
    mloss = float(rast.mask_loss().item())
    tg = [scenes.target_image(c.height, c.width, seed=60 + k) for k, c in enumerate(cams)]
    torch.cuda.synchronize()
    gimg = img.cpu().numpy()
    so = rast.splat_outputs()
    mask = so["mask"].cpu().numpy()
    po = 0
    t0 = 0
    dimgs = []
    orc = []
    for k, (s, cam) in enumerate(zip(sc, cams)):
        ocfg = pipeline.OracleConfig(bg=cfg.bg, seed=cfg.seed, iteration=cfg.iteration,
                                     index_offset=int(offs[k]), eps=1e-4, lambda_m=lambda_m)
        views, M, minfo = pipeline.forward(s, [cam], ocfg)
        v = views[0]
        assert np.array_equal(mask[offs[k]:offs[k] + sizes[k]], M)
        assert int(so["mask_count"][k].item()) == int(M.sum())
        mloss -= pipeline.mask_loss(M, ocfg)
        gx, gy = v.fp32["grid"]
        lists = _tile_lists(rast, t0, gx * gy, int(offs[k]))
        for t, lst in enumerate(lists):
            s0, e0 = v.ranges[t]
            assert np.array_equal(lst, v.sorted_vals[s0:e0].astype(np.int64)), (k, t)
        n = 3 * cam.width * cam.height
        im = gimg[po:po + n].reshape(3, cam.height, cam.width)
        straddle = (v.out["flags"] & 11) != 0
        d = np.abs(im - v.out["image"]).max(0)
        assert not ((d > 2e-4) & ~straddle).any()
        _, dg = pipeline.l1_loss_grad(v.out["image"], tg[k])
        dg = dg * (~straddle)[None]
        dimgs.append(dg)
        orc.append((s, cam, ocfg, views, M, minfo, dg))
        po += n
        t0 += gx * gy
    assert abs(mloss) < 1e-6                      # sum over scenes of lambda_m L_m
    flat = np.concatenate([d.reshape(-1) for d in dimgs]).astype(np.float32)
    out = rast.backward(torch.as_tensor(flat).cuda())
    torch.cuda.synchronize()
    for k, (s, cam, ocfg, views, M, minfo, dg) in enumerate(orc):
        grads, _ = pipeline.backward(s, [cam], ocfg, views, M, minfo, [dg])
        sl = slice(int(offs[k]), int(offs[k]) + sizes[k])
        for name in ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits"):
            e = rel_l2(out[name][sl].cpu().numpy(), grads[name])
            assert e < 1e-3, (k, name, e)


def test_autotuner_picks_and_caches(tmp_path, monkeypatch):
    """The autotuner chooses the tile shape, the sort digit width and both
    staging depths, records all of them (with every timing it took) in the
    cache, and returns the cached choice on the next call."""
    import json
    from paper_2412_20522_gb300 import autotune
    monkeypatch.setenv("MASKGS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    g, cams, tgt = scenes.tiny_workload(8000)
    p = to_device(g)
    t = torch.as_tensor(tgt).cuda().reshape(-1)
    best = autotune.autotune(p, cams, t, steps=2)
    assert (best.tile_w, best.tile_h) in autotune.TILE_SHAPES
    assert best.sort in autotune.SORTS
    assert best.render_batch in autotune.FWD_BATCHES
    assert best.render_batch_bwd in autotune.BWD_BATCHES
    entry = next(iter(json.load(open(tmp_path / "tune.json")).values()))
    assert all(k in entry for k in autotune.TUNED)
    assert len(entry["ms"]) >= len(autotune.TILE_SHAPES) + 3
    again = autotune.autotune(p, cams, t, steps=2)                    # from the cache
    assert all(getattr(again, k) == getattr(best, k) for k in autotune.TUNED)
    assert autotune.autotune_tile(p, cams, t) == (best.tile_w, best.tile_h)


def test_l1_loss_grad_views_at_every_alignment():
    """dL/dimage = sign(C - target) / (3 W H) per view, sign(0) = 0, and the
    summed per-view mean |C - target|, for views whose offsets leave each of
    the four 16-byte alignments (vector body, scalar head and tail)."""
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import make_views
    sizes = [(5, 3), (7, 5), (33, 17), (2, 1), (64, 48)]
    cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), w, h, 30.0) for w, h in sizes]
    n = sum(3 * w * h for w, h in sizes)
    rng = np.random.default_rng(3)
    img = rng.random(n).astype(np.float32)
    tgt = rng.random(n).astype(np.float32)
    tgt[::7] = img[::7]                                   # exact zeros of the difference
    views = make_views(cams, [(0, 1)] * len(cams))
    gi, gt = torch.as_tensor(img).cuda(), torch.as_tensor(tgt).cuda()
    grad = torch.full((n,), 7.0, device="cuda")
    loss = torch.zeros(1, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    import ctypes as C
    abi.mg_l1_loss_grad(gi, gt, views, len(cams), grad, loss, C.c_void_p(stream))
    torch.cuda.synchronize()
    exp = np.empty(n, np.float32)
    o = 0
    tot = 0.0
    for w, h in sizes:
        m = 3 * w * h
        d = img[o:o + m] - tgt[o:o + m]
        inv = np.float32(1.0) / np.float32(m)
        exp[o:o + m] = np.where(d > 0, inv, np.where(d < 0, -inv, np.float32(0.0)))
        tot += float(np.abs(d.astype(np.float64)).mean())
        o += m
    assert np.array_equal(grad.cpu().numpy(), exp)
    assert float(loss.item()) == pytest.approx(tot, rel=1e-5)
