"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on seeded inputs.

Bit-exact: masks, tile counts, radii, 2D means and depth keys, instance
offsets and count, sorted keys and values, tile ranges.  Floating point:
images within 2e-4 absolute per channel and gradients within 1e-3 relative L2
per tensor (FP32 against FP64).  Pixels where one FP64 fragment decision lies
within the straddle band of its threshold (alpha floor, termination, power
sign) are counted and reported; they are excluded from the image bound only
if flagged, and their upstream gradient is zeroed on both sides.
"""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2, split_views, to_device
from oracle import binning, pipeline
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 2e-4
GRAD_TOL = 1e-3
EPS = 1e-4          # straddle band (relative), see the oracle's render


@pytest.fixture(scope="module")
def rz():
    from paper_2412_20522_gb300 import rasterize
    return rasterize


def _run(rz, g, cams, targets, cfg_kw=None, tile=(16, 16), view_ranges=None, capacity=0):
    cfg_kw = cfg_kw or {}
    dev = to_device(g)
    rcfg = rz.RasterConfig(tile_w=tile[0], tile_h=tile[1], **cfg_kw)
    rast = rz.Rasterizer(capacity=capacity)
    img = rast.forward(dev, cams, rcfg, view_ranges=view_ranges, count_fragments=True)
    torch.cuda.synchronize()
    return rast, dev, img


# launch choices of the GPU path that change no result the oracle defines
LAUNCH_ONLY = ("sort", "render_batch", "render_batch_bwd")


def _oracle(g, cams, cfg_kw=None, tile=(16, 16)):
    cfg_kw = {k: v for k, v in (cfg_kw or {}).items() if k not in LAUNCH_ONLY}
    gm = cfg_kw.pop("given_mask", None)
    ocfg = pipeline.OracleConfig(tile_w=tile[0], tile_h=tile[1], eps=EPS, **cfg_kw)
    if gm is not None:
        ocfg.given_mask = gm.cpu().numpy()
    views, M, minfo = pipeline.forward(g, cams, ocfg)
    return ocfg, views, M, minfo


def _check_discrete(rast, views, M, cams):
    so = rast.splat_outputs()
    assert np.array_equal(so["mask"].cpu().numpy(), M), "sampled masks differ"
    # depth order of all records (all views), and the scan in that order; the
    # bucket sort needs no depth order: its scan runs in record order
    tiles_all = np.concatenate([v.fp32["tiles"] for v in views]).astype(np.int64)
    if so["order"] is None:
        order = np.arange(tiles_all.size)
    else:
        order = binning.depth_order(np.concatenate([v.fp32["depth_bits"] for v in views]),
                                    np.concatenate([v.fp32["tiles"] > 0 for v in views]))
        assert np.array_equal(so["order"].cpu().numpy().view(np.uint32), order), \
            "depth order differs"
    exp_off = np.concatenate([[0], np.cumsum(tiles_all[order])[:-1]]) if order.size else order
    assert np.array_equal(so["offsets"].cpu().numpy().view(np.uint32).astype(np.int64), exp_off), \
        "scan offsets differ"
    rec = so["record"].cpu().numpy()
    tiles = so["tiles"].cpu().numpy().view(np.uint32)
    radius = so["radius"].cpu().numpy()
    K_gpu = int(so["num_instances"].item())               # rectangle instances
    Ks_gpu = int(so["num_sorted"].item())                 # kept by the tile filter
    R0 = 0
    T0 = 0
    K0 = 0
    Kc = 0
    ranges = so["ranges"].cpu().numpy().view(np.uint32).reshape(-1, 2)
    vals = so["sorted_vals"].cpu().numpy().view(np.uint32)[:Ks_gpu]
    keys = rast.sorted_keys().cpu().numpy().view(np.uint32)[:Ks_gpu]
    for v, cam in zip(views, cams):
        n = v.fp32["tiles"].shape[0]
        fp = v.fp32
        assert np.array_equal(tiles[R0:R0 + n], fp["tiles"]), "tiles_touched differ"
        assert np.array_equal(radius[R0:R0 + n], fp["radius"]), "radius differs"
        vis = fp["visible"]
        r = rec[R0:R0 + n]
        assert np.array_equal(r[vis, 0].view(np.uint32), fp["px"][vis].view(np.uint32))
        assert np.array_equal(r[vis, 1].view(np.uint32), fp["py"][vis].view(np.uint32))
        assert np.array_equal(r[vis, 11].view(np.uint32), fp["depth_bits"][vis])
        nt = v.ranges.shape[0]
        # instance keys are global tile ids: the oracle's tile of view v plus T0
        otiles = (v.sorted_keys >> np.uint64(32)).astype(np.int64) + T0
        assert np.array_equal(keys[K0:K0 + v.K_kept].astype(np.int64), otiles), "sorted tiles differ"
        assert np.array_equal(vals[K0:K0 + v.K_kept], v.sorted_vals.astype(np.uint32) + R0), \
            "sorted values differ"
        gr = ranges[T0:T0 + nt].astype(np.int64)
        orr = v.ranges.astype(np.int64)
        nonempty = orr[:, 1] > orr[:, 0]
        assert np.array_equal(gr[nonempty], orr[nonempty] + K0), "tile ranges differ"
        assert (gr[~nonempty, 1] == gr[~nonempty, 0]).all()
        R0 += n
        T0 += nt
        K0 += v.K_kept
        Kc += v.K
    assert K_gpu == Kc
    assert Ks_gpu == K0


def _check_images(rast, img, views, cams, report):
    so = rast.splat_outputs()
    gimgs = split_views(img.cpu().numpy(), cams)
    gT = split_views(so["final_T"].cpu().numpy(), cams, 1)
    gN = split_views(so["n_contrib"].cpu().numpy(), cams, 1)
    masks = []
    for v, gi, gt, gn in zip(views, gimgs, gT, gN):
        straddle = (v.out["flags"] & 11) != 0
        d = np.abs(gi - v.out["image"]).max(0)
        bad = (d > IMG_TOL) & ~straddle
        report.append(dict(pixels=d.size, straddle=int(straddle.sum()),
                           over_tol=int((d > IMG_TOL).sum()), max_err_clean=float(d[~straddle].max()) if (~straddle).any() else 0.0))
        assert not bad.any(), f"{bad.sum()} non-straddle pixels over {IMG_TOL}: max {d[bad].max()}"
        assert np.abs(gt - v.out["final_T"])[~straddle].max() < 1e-4
        assert np.array_equal(gn[~straddle], v.out["n_contrib"][~straddle])
        assert straddle.mean() < 0.02
        masks.append(straddle)
    return masks


def _check_backward(rast, dev, g, cams, ocfg, views, M, minfo, straddles, targets):
    # the same upstream gradient on both sides: the oracle's L1 gradient,
    # zeroed on straddle pixels
    dimgs = []
    for v, t, s in zip(views, targets, straddles):
        _, d = pipeline.l1_loss_grad(v.out["image"], t)
        d = d * (~s)[None]
        dimgs.append(d)
    grads, per_view = pipeline.backward(g, cams, ocfg, views, M, minfo, dimgs)
    flat = np.concatenate([d.reshape(-1) for d in dimgs]).astype(np.float32)
    out = rast.backward(torch.as_tensor(flat).cuda())
    torch.cuda.synchronize()
    errs = {}
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits"):
        errs[k] = rel_l2(out[k].cpu().numpy(), grads[k])
    g2 = rast.splat_outputs()["grad2d"].cpu().numpy().reshape(-1, 12)
    R0 = 0
    for v, pv in zip(views, per_view):
        n = pv["dmask"].shape[0]
        G = g2[R0:R0 + n]
        errs.setdefault("dmean2d", []).append(rel_l2(G[:, 0:2], pv["dmean2d"]))
        errs.setdefault("dconic", []).append(rel_l2(G[:, 2:5], pv["dconic"]))
        errs.setdefault("dopacity", []).append(rel_l2(G[:, 5], pv["dopacity"]))
        errs.setdefault("drgb", []).append(rel_l2(G[:, 6:9], pv["drgb"]))
        errs.setdefault("dmask", []).append(rel_l2(G[:, 9], pv["dmask"]))
        R0 += n
    flatten = {k: (max(v) if isinstance(v, list) else v) for k, v in errs.items()}
    bad = {k: e for k, e in flatten.items() if not e <= GRAD_TOL}
    assert not bad, f"gradients over {GRAD_TOL} relative L2: {bad} (all: {flatten})"
    return flatten


def _full_check(rz, g, cams, targets, cfg_kw=None, tile=(16, 16), capacity=0):
    rast, dev, img = _run(rz, g, cams, targets, cfg_kw, tile, capacity=capacity)
    ocfg, views, M, minfo = _oracle(g, cams, cfg_kw, tile)
    _check_discrete(rast, views, M, cams)
    rep = []
    straddles = _check_images(rast, img, views, cams, rep)
    errs = _check_backward(rast, dev, g, cams, ocfg, views, M, minfo, straddles, targets)
    print("image report", rep, "grad errors", errs)
    return rast, views


def test_tiny_workload(rz):
    g, cams, tgt = scenes.tiny_workload()
    _full_check(rz, g, cams, [tgt])


def test_tiny_workload_background_and_other_seed(rz):
    g, cams, tgt = scenes.tiny_workload()
    _full_check(rz, g, cams, [tgt], dict(bg=(0.9, 0.4, 0.1), seed=77, iteration=12345678901))


def test_whole_rectangle_tile_lists(rz):
    """bin_mode MG_BIN_RECT: the 3DGS lists (whole 3-sigma rectangles, no tile
    filter) -- same images and gradients, longer lists."""
    g, cams, tgt = scenes.tiny_workload()
    _full_check(rz, g, cams, [tgt], dict(bin_mode=1, bg=(0.3, 0.2, 0.1)))
    g = scenes.cluster_gaussians(40_000, seed=8)
    cams = [scenes.ring_camera(0.0, 4.0, 200, 130, 150.0)]
    _full_check(rz, g, cams, [scenes.target_image(130, 200, seed=2)], dict(bin_mode=1))


def test_tile_8x32_and_ragged_frame(rz):
    g = scenes.uniform_gaussians(3000, seed=5)
    cams = [scenes.look_at_camera((0.2, -0.1, -3.2), (0, 0, 0), 100, 75, 90.0)]
    tgt = scenes.target_image(75, 100, seed=9)
    for tile in ((8, 32), (32, 8), (16, 16)):
        _full_check(rz, g, cams, [tgt], dict(bg=(0.2, 0.3, 0.4)), tile)


def test_all_ones_and_given_masks(rz):
    g, cams, tgt = scenes.tiny_workload(4000)
    _full_check(rz, g, cams, [tgt], dict(mask_mode=1))
    gm = torch.as_tensor((np.arange(g.n) % 3 == 0).astype(np.uint8)).cuda()
    _full_check(rz, g, cams, [tgt], dict(mask_mode=2, given_mask=gm))


def test_sh_degrees(rz):
    for deg in (0, 1, 2):
        g = scenes.uniform_gaussians(2000, seed=3 + deg, sh_degree=deg)
        cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 64, 48, 60.0)]
        _full_check(rz, g, cams, [scenes.target_image(48, 64, seed=4)])


def test_multi_view_shared_mask(rz):
    g = scenes.cluster_gaussians(20_000, seed=21, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(2 * math.pi * k / 3, 4.0, 96 + 16 * k, 64 + 8 * k, 80.0)
            for k in range(3)]
    tg = [scenes.target_image(c.height, c.width, seed=30 + k) for k, c in enumerate(cams)]
    _full_check(rz, g, cams, tg, dict(bg=(0.1, 0.1, 0.1)))


def test_mid_scene_clusters(rz):
    """100k clustered Gaussians, camera inside the cloud: needle splats, huge
    near-camera splats, long tile lists, many tiles with a ragged edge."""
    g = scenes.cluster_gaussians(100_000, seed=8)
    cams = [scenes.ring_camera(0.0, 4.0, 389, 259, 287.5)]
    _full_check(rz, g, cams, [scenes.target_image(259, 389, seed=2)])


def test_empty_scene_renders_background(rz):
    g = scenes.uniform_gaussians(0)
    cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 40, 30, 30.0)]
    rast, dev, img = _run(rz, g, cams, None, dict(bg=(0.25, 0.5, 0.75)))
    im = img.cpu().numpy().reshape(3, 30, 40)
    assert np.allclose(im[0], 0.25) and np.allclose(im[1], 0.5) and np.allclose(im[2], 0.75)
    assert (rast.splat_outputs()["final_T"].cpu().numpy() == 1.0).all()


def test_all_culled_scene(rz):
    g = scenes.uniform_gaussians(500, seed=1)
    g.means[:, 2] = -10.0                      # every Gaussian behind the camera
    cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 48, 48, 40.0)]
    rast, dev, img = _run(rz, g, cams, None)
    assert int(rast.num_instances.item()) == 0
    assert np.allclose(img.cpu().numpy(), 0.0)
    out = rast.backward(torch.ones_like(img))
    for k in ("means", "sh", "opacity_logit"):
        assert float(out[k].abs().max()) == 0.0


def _degenerate_scene():
    """A small cloud plus the method's corner cases, each placed at a chosen
    pixel and camera depth (input placement only)."""
    g = scenes.uniform_gaussians(2000, seed=41)
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 96, 80, 80.0)
    Rm = cam.viewmat[:, :3].astype(np.float64)
    tv = cam.viewmat[:, 3].astype(np.float64)

    def world(u, v, z):
        t = np.array([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z])
        return Rm.T @ (t - tv)

    rows = []          # (mean, scale, opacity logit)
    # an opaque stack on one pixel centre: 8 depths x 5 exact copies (depth
    # ties broken by index), opacity ~1 (alpha clamped at 0.99), the pixel
    # terminating after two blends
    for k in range(8):
        for _ in range(5):
            rows.append((world(40.5, 36.5, 2.0 + 0.1 * k), 0.03, 9.0))
    rows.append((world(48.0, 40.0, 3.0), 2.5, -1.0))          # covers every tile
    for u in (16, 32, 48, 64, 80):                            # on tile corners
        for v in (16, 32, 48, 64):
            rows.append((world(u, v, 2.5), 0.01, 2.0))
    for k in range(10):                                       # opacity under 1/255
        rows.append((world(10.0 + 7 * k, 70.0, 2.2), 0.05, -7.0))
    rows.append((world(60.0, 20.0, 0.2005), 0.002, 1.0))      # just past the near plane
    rows.append((world(62.0, 22.0, 0.1995), 0.002, 1.0))      # just before it: culled
    m = len(rows)
    g.means[:m] = np.array([r[0] for r in rows], np.float32)
    g.log_scales[:m] = np.log(np.array([[r[1]] * 3 for r in rows], np.float64)).astype(np.float32)
    g.opacity_logit[:m] = np.array([r[2] for r in rows], np.float32)
    return g, [cam]


def test_degenerate_cases(rz):
    """Early termination, the 0.99 clamp, exact depth ties, a frame-filling
    splat, splats on tile corners, opacities under the floor and the near
    plane, against the oracle."""
    g, cams = _degenerate_scene()
    tgt = scenes.target_image(80, 96, seed=43)
    rast, views = _full_check(rz, g, cams, [tgt], dict(bg=(0.2, 0.4, 0.6)))
    fp = views[0].fp32
    assert fp["visible"][40] and fp["rect_tiles"][40] == 30     # the frame-filling splat
    assert fp["visible"][71] and not fp["visible"][72]          # the near plane
    final_T = rast.splat_outputs()["final_T"].cpu().numpy().reshape(80, 96)
    assert final_T[36, 40] <= 0.0101                            # one clamped blend, then stop


@pytest.mark.parametrize("wh", [(1, 1), (17, 1), (3, 2), (1, 33)])
def test_frames_smaller_than_a_tile(rz, wh):
    """Frames of a few pixels: one tile (or a row of them) with most of its
    pixels outside the frame; every warp block is partly or wholly outside."""
    w, h = wh
    g = scenes.uniform_gaussians(2000, seed=71)
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), w, h, 40.0)
    _full_check(rz, g, [cam], [scenes.target_image(h, w, seed=72)], dict(bg=(0.1, 0.5, 0.3)))


def test_every_gaussian_masked(rz):
    """M = 0 everywhere: the image is the background and only dL/dM (hence
    the mask scores' gradient) is non-zero."""
    g, cams, tgt = scenes.tiny_workload(3000)
    gm = torch.zeros(g.n, dtype=torch.uint8, device="cuda")
    rast, _ = _full_check(rz, g, cams, [tgt], dict(mask_mode=2, given_mask=gm,
                                                   bg=(0.3, 0.6, 0.9)))
    img = rast.forward(to_device(g), cams, rz.RasterConfig(mask_mode=2, given_mask=gm,
                                                           bg=(0.3, 0.6, 0.9)))
    torch.cuda.synchronize()
    im = img.cpu().numpy().reshape(3, -1)
    for c, b in enumerate((0.3, 0.6, 0.9)):
        assert np.all(im[c] == np.float32(b))


def test_duplication_chunks_inside_large_splats(rz):
    """Frame-filling splats whose instance ranges cross several 512-slot
    duplication chunks (the scan marks each chunk's owning splat), with the
    instance buffer sized to the exact count (the last chunk ends at the
    capacity), against the oracle."""
    g = scenes.uniform_gaussians(3000, seed=61)
    cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 1000, 760, 600.0)
    for k in range(4):                          # low-opacity splats over the whole frame
        g.means[k] = (0.05 * k, -0.04 * k, 0.1 * k)
        g.log_scales[k] = np.log(2.5)
        g.opacity_logit[k] = -2.0 - 0.5 * k
    tgt = scenes.target_image(760, 1000, seed=62)
    first = rz.Rasterizer()
    first.forward(to_device(g), [cam], rz.RasterConfig(), check=True)
    torch.cuda.synchronize()
    K = int(first.num_instances.item())
    assert K > 4 * 3000                         # each large splat spans several chunks
    rast, views = _full_check(rz, g, [cam], [tgt], capacity=K)
    assert rast.capacity == K                   # no regrowth: the exact size sufficed
    assert int(rast.num_instances.item()) == K
