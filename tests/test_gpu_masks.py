"""GPU parity of the mask loss (Sec. 3.5, Eq. 7-8), the ablations of Sec. 4.3
(threshold mask with a straight-through sigmoid; mask multiplied into the
opacity), the pruning sampler and compaction (Sec. 3.5) and the forward-only
inference renderer -- through the C ABI, against the oracle.  Discrete
outputs (masks, keep flags, survivor rows, indices, counts) bit for bit."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2, to_device
from oracle import pipeline, pruning
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rz():
    from paper_2412_20522_gb300 import rasterize
    return rasterize


def _full(rz, g, cams, tg, cfg_kw):
    from test_gpu_parity import _full_check
    return _full_check(rz, g, cams, tg, cfg_kw)


@pytest.mark.parametrize("kind", [0, 1])
def test_mask_loss_gumbel(rz, kind):
    g, cams, tgt = scenes.tiny_workload(6000)
    kw = dict(lambda_m=0.25, mask_loss=kind, bg=(0.1, 0.2, 0.3))
    rast, views = _full(rz, g, cams, [tgt], kw)
    so = rast.splat_outputs()
    M = so["mask"].cpu().numpy()
    assert int(so["mask_count"][0].item()) == int(M.sum())
    ocfg = pipeline.OracleConfig(**kw)
    assert float(rast.mask_loss().item()) == pytest.approx(pipeline.mask_loss(M, ocfg), rel=1e-6)


def test_mask_loss_changes_only_mask_logit_gradients(rz):
    """lambda_m enters dL/dM only: every other gradient is unchanged, and the
    mask-logit gradients move by the straight-through factor times the
    closed-form 2 lambda_m k / N^2."""
    g, cams, tgt = scenes.tiny_workload(4000)
    p = to_device(g)
    t = torch.as_tensor(tgt).cuda().reshape(-1)
    outs = []
    for lam in (0.0, 0.5):
        rast = rz.Rasterizer()
        img = rast.forward(p, cams, rz.RasterConfig(lambda_m=lam))
        loss, dimg = rast.l1_loss_grad(img, t)
        outs.append((rast.backward(dimg), rast.splat_outputs(), float(loss)))
    torch.cuda.synchronize()
    (a, so, l0), (b, _, l1) = outs
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert rel_l2(b[k].cpu().numpy(), a[k].cpu().numpy()) < 1e-5, k
    M = so["mask"].cpu().numpy().astype(np.float64)
    y0 = so["mask_soft"].cpu().numpy().astype(np.float64)
    n = M.size
    extra = 2 * 0.5 * M.sum() / n / n * y0 * (1 - y0)
    d = (b["mask_logits"] - a["mask_logits"]).cpu().numpy()[:, 0]
    assert np.allclose(d, extra, rtol=1e-3, atol=1e-9)
    assert l1 - l0 == pytest.approx(0.5 * (M.sum() / n) ** 2, rel=1e-5)


@pytest.mark.parametrize("theta", [0.5, 0.01])
def test_ste_threshold_mask(rz, theta):
    g, cams, tgt = scenes.tiny_workload(6000)
    kw = dict(mask_mode=3, ste_logit=rz.RasterConfig.ste_logit_of(theta), lambda_m=0.1)
    _full(rz, g, cams, [tgt], kw)


def test_opacity_ablation(rz):
    g, cams, tgt = scenes.tiny_workload(6000)
    _full(rz, g, cams, [tgt], dict(mask_apply=1, bg=(0.2, 0.1, 0.0)))
    _full(rz, g, cams, [tgt], dict(mask_apply=1, mask_mode=3, ste_logit=0.0, lambda_m=0.2))


def test_opacity_ablation_image_equals_masked_rasterisation(rz):
    """Two ways of removing a Gaussian from the blend give the same image bit
    for bit on the GPU too; only the mask-logit gradients differ."""
    g = scenes.cluster_gaussians(50_000, seed=12, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.3, 4.0, 200, 150, 180.0)]
    p = to_device(g)
    imgs = []
    for apply in (0, 1):
        rast = rz.Rasterizer()
        imgs.append(rast.forward(p, cams, rz.RasterConfig(mask_apply=apply)).clone())
    torch.cuda.synchronize()
    assert torch.equal(imgs[0], imgs[1])


def _logits(n, seed):
    rng = np.random.default_rng(seed)
    l = np.empty((n, 2), np.float32)
    l[:, 0] = rng.normal(-2.0, 1.5, n)
    l[:, 1] = rng.normal(0.0, 1.0, n)
    return l


@pytest.mark.parametrize("n,draws", [(1, 10), (4097, 10), (300_001, 10), (300_001, 1)])
def test_prune_sample_bit_exact(n, draws):
    from paper_2412_20522_gb300 import prune
    g = scenes.uniform_gaussians(n, seed=n % 97)
    g.mask_logits = _logits(n, 5)
    keep = prune.prune_sample(to_device(g), seed=123, iteration=456, n_draws=draws)
    ref = pruning.keep_mask(g.mask_logits, 123, 456, draws)
    got = keep.cpu().numpy()
    assert np.array_equal(got, ref)
    if n > 1000:
        assert 0.05 < got.mean() < 0.95


def _check_compact(p, keep_np):
    from paper_2412_20522_gb300 import prune
    c = prune.Compactor()
    c.run(p, torch.as_tensor(keep_np).cuda())
    out, new_index = c.result()
    def rows_as_bytes(t):
        t = t.cpu()
        width = int(np.prod(t.shape[1:])) if t.dim() > 1 else 1
        return t.reshape(t.shape[0], width).contiguous().view(torch.uint8).numpy()

    ref, ref_index, cnt = pruning.compact({k: rows_as_bytes(v) for k, v in p.items()}, keep_np)
    assert int(c.n_kept.item()) == cnt
    assert np.array_equal(new_index.cpu().numpy(), ref_index)
    for k, v in out.items():
        got = rows_as_bytes(v)
        assert got.shape == ref[k].shape, k
        assert np.array_equal(got, ref[k]), k


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("deg", [3, 0])
def test_compact_bit_exact(dtype, deg):
    stored = ("log_scales", "quats", "opacity_logit", "sh")
    for n in (1, 4095, 4096, 4097, 250_003):
        g = scenes.uniform_gaussians(n, seed=n % 13, sh_degree=deg)
        p = {k: (v.to(dtype) if k in stored else v) for k, v in to_device(g).items()}
        rng = np.random.default_rng(n)
        for keep in ((rng.random(n) < 0.4), np.zeros(n, bool), np.ones(n, bool),
                     (np.arange(n) % 2 == 0)):
            _check_compact(p, keep.astype(np.uint8))


def test_compact_offset_rows_use_narrower_words():
    """Arrays that start one row in (12-byte means, 6-byte BF16 scales ...)
    take the widest word their alignment allows; the result is the same."""
    g = scenes.uniform_gaussians(10_001, seed=2)
    stored = ("log_scales", "quats", "opacity_logit", "sh")
    full = {k: (v.to(torch.bfloat16) if k in stored else v) for k, v in to_device(g).items()}
    p = {k: v[1:] for k, v in full.items()}
    keep = (np.random.default_rng(1).random(10_000) < 0.5).astype(np.uint8)
    _check_compact(p, keep)


def test_inference_render_of_pruned_model(rz):
    """The pruned model's inference image equals, bit for bit, the training
    forward of the full model with the keep flags as a given mask (a masked
    Gaussian leaves the blend exactly as a deleted one, Eq. 3-4), and the
    inference image of the full model equals its all-ones training forward."""
    from paper_2412_20522_gb300 import prune
    g = scenes.cluster_gaussians(80_000, seed=14, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    g.mask_logits = _logits(g.n, 9)
    cams = [scenes.ring_camera(0.9, 4.0, 256, 192, 220.0),
            scenes.ring_camera(2.0, 4.0, 160, 120, 140.0)]
    p = to_device(g)
    cfg = rz.RasterConfig(bg=(0.05, 0.1, 0.2))
    small, new_index, keep = prune.prune(p, seed=1, iteration=2, n_draws=10)
    assert 0 < small["means"].shape[0] < g.n
    r1 = rz.Rasterizer()
    inf = r1.forward(small, cams, cfg, inference=True).clone()
    r2 = rz.Rasterizer()
    given = r2.forward(p, cams, rz.RasterConfig(bg=cfg.bg, mask_mode=2, given_mask=keep)).clone()
    r3 = rz.Rasterizer()
    inf_full = r3.forward(p, cams, cfg, inference=True).clone()
    r4 = rz.Rasterizer()
    ones = r4.forward(p, cams, rz.RasterConfig(bg=cfg.bg, mask_mode=1)).clone()
    torch.cuda.synchronize()
    assert torch.equal(inf, given)
    assert torch.equal(inf_full, ones)


def test_inference_render_matches_plain_3dgs_oracle(rz):
    from test_gpu_parity import EPS
    g, cams, _ = scenes.tiny_workload(5000)
    rast = rz.Rasterizer()
    img = rast.forward(to_device(g), cams, rz.RasterConfig(bg=(0.3, 0.3, 0.3)), inference=True)
    torch.cuda.synchronize()
    ocfg = pipeline.OracleConfig(bg=(0.3, 0.3, 0.3), mask_mode=pipeline.MASK_ALL_ONES, eps=EPS)
    views, _, _ = pipeline.forward(g, cams, ocfg)
    v = views[0]
    im = img.cpu().numpy().reshape(3, cams[0].height, cams[0].width)
    straddle = (v.out["flags"] & 11) != 0
    d = np.abs(im - v.out["image"]).max(0)
    assert not ((d > 2e-4) & ~straddle).any()
