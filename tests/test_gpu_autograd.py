"""The differentiable pass through torch autograd (Sec. 3.3: sampling and
rendering are both differentiable, so the existence scores receive gradients
through Eq. 6).

``rasterize()`` (the ``torch.autograd.Function`` over the hand-written
backward) -> L1 render loss + lambda_m L_m (Eq. 7-8) -> ``loss.backward()``,
and every parameter's ``.grad`` against the FP64 oracle's gradient of the same
loss.  Straddle pixels (an FP64 fragment decision within the band of its
threshold) and pixels whose L1 sign differs between the GPU and the oracle
image carry no weight in the loss, on both sides.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import PARAMS, rel_l2, to_device
from oracle import pipeline
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
EPS = 1e-4
# two GPU runs of the same gradient: float-atomic summation order differs
ATOMIC_TOL = 1e-4


def _workload(which):
    if which == "tiny":
        g, cams, tgt = scenes.tiny_workload()
        return g, cams, [tgt], (0.0, 0.0, 0.0)
    g = scenes.cluster_gaussians(100_000, seed=8)
    cams = [scenes.ring_camera(0.0, 4.0, 389, 259, 287.5)]
    return g, cams, [scenes.target_image(259, 389, seed=2)], (0.2, 0.3, 0.1)


def _leaf_params(g):
    return {k: v.clone().requires_grad_(True) for k, v in to_device(g).items()}


@pytest.mark.parametrize("which", ["tiny", "clusters100k"])
def test_autograd_step_matches_oracle(which):
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer, rasterize
    g, cams, tgts, bg = _workload(which)
    lam = 0.1
    ocfg = pipeline.OracleConfig(eps=EPS, lambda_m=lam, bg=bg)
    views, M, minfo = pipeline.forward(g, cams, ocfg)

    params = _leaf_params(g)
    cfg = RasterConfig(lambda_m=lam, bg=bg)
    imgs, ml = rasterize(params, cams, cfg, return_mask_loss=True)
    weights, dimgs = [], []
    for img, v, t in zip(imgs, views, tgts):
        straddle = (v.out["flags"] & 11) != 0
        sg = np.sign(img.detach().cpu().numpy().astype(np.float64) - t)
        so = np.sign(v.out["image"] - t)
        w = (~straddle)[None] & (sg == so)
        assert (sg != so)[:, ~straddle].mean() < 1e-3
        weights.append(torch.as_tensor(w.astype(np.float32)).cuda())
        dimgs.append(so * w / so.size)
    tt = [torch.as_tensor(t).cuda() for t in tgts]
    loss = sum((w * (i - t).abs()).sum() / i.numel() for w, i, t in zip(weights, imgs, tt)) + ml
    loss.backward()
    torch.cuda.synchronize()

    # the oracle: the same weighted L1 plus lambda_m L_m (added by its backward)
    ref, _ = pipeline.backward(g, cams, ocfg, views, M, minfo, dimgs)
    assert abs(float(ml.item()) - pipeline.mask_loss(M, ocfg)) < 1e-6
    errs = {k: rel_l2(params[k].grad.cpu().numpy(), ref[k]) for k in PARAMS}
    print(which, "autograd grad rel L2", errs)
    assert all(e <= GRAD_TOL for e in errs.values()), errs

    # the same gradients through the plain C-ABI sequence (no autograd), to
    # the rounding of float atomics (their order differs from run to run, and
    # the chain to scales and rotations of thin splats magnifies it)
    rast = Rasterizer()
    rast.forward({k: p.detach() for k, p in params.items()}, cams, cfg)
    flat = torch.as_tensor(np.concatenate([d.reshape(-1) for d in dimgs]).astype(np.float32))
    direct = rast.backward(flat.cuda())
    torch.cuda.synchronize()
    for k in PARAMS:
        e = rel_l2(params[k].grad.cpu().numpy(), direct[k].cpu().numpy())
        assert e <= ATOMIC_TOL, (k, e)


def test_two_pending_forwards_on_one_rasterizer():
    """Two views rendered by separate rasterize() calls on one Rasterizer,
    both forwards before either backward: each backward reads its own
    forward's state, so the summed gradients equal those of the two views'
    backwards taken one after the other through the plain sequence."""
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer, rasterize
    g = scenes.cluster_gaussians(30_000, seed=12, centre_radius=1.5, reject_radius=2.0,
                                 log_scale_mu=-4.0, log_scale_sigma=0.5)
    cams = [scenes.ring_camera(0.3, 4.0, 160, 120, 130.0),
            scenes.ring_camera(2.0, 4.0, 128, 96, 110.0)]
    tgts = [torch.as_tensor(scenes.target_image(c.height, c.width, seed=40 + k)).cuda()
            for k, c in enumerate(cams)]
    cfg = RasterConfig(bg=(0.1, 0.2, 0.3), lambda_m=0.05)
    params = _leaf_params(g)
    rast = Rasterizer()
    a, mla = rasterize(params, [cams[0]], cfg, rast, return_mask_loss=True)
    b = rasterize(params, [cams[1]], cfg, rast)            # overwrites rast's buffers
    # an inference forward in between must not disturb either pending state
    rast.forward({k: p.detach() for k, p in params.items()}, [cams[1]], cfg, inference=True)
    loss = (a[0] - tgts[0]).abs().mean() + 0.5 * (b[0] - tgts[1]).abs().mean() + 2.0 * mla
    loss.backward()
    torch.cuda.synchronize()

    det = {k: p.detach() for k, p in params.items()}
    ref = {k: torch.zeros(p.shape, dtype=torch.float64) for k, p in det.items()}
    for cam, t, scale, lam in ((cams[0], tgts[0], 1.0, 2.0 * cfg.lambda_m),
                               (cams[1], tgts[1], 0.5, 0.0)):
        r = Rasterizer()
        img = r.forward(det, [cam], cfg)
        d = torch.sign(img.view(3, cam.height, cam.width) - t) * (scale / img.numel())
        out = r.backward(d.reshape(-1).contiguous(), lambda_m=lam)
        for k in ref:
            ref[k] += out[k].double().cpu()
    torch.cuda.synchronize()
    for k in PARAMS:
        e = rel_l2(params[k].grad.cpu().numpy(), ref[k].numpy())
        assert e <= ATOMIC_TOL, (k, e)


def test_autograd_reduced_storage_returns_parameter_dtype():
    """BF16 attribute storage: the gradients reach autograd in the parameters'
    dtype, and equal (to BF16 rounding) the FP32 gradients of the plain
    sequence on the same stored values."""
    from paper_2412_20522_gb300.rasterize import STORED, RasterConfig, Rasterizer, rasterize
    g, cams, tgt = scenes.tiny_workload(4000)
    base = to_device(g)
    params = {k: (v.to(torch.bfloat16) if k in STORED else v).clone().requires_grad_(True)
              for k, v in base.items()}
    t = torch.as_tensor(tgt).cuda()
    img = rasterize(params, cams, RasterConfig())[0]
    (img - t).abs().mean().backward()
    torch.cuda.synchronize()
    r = Rasterizer()
    im2 = r.forward({k: p.detach() for k, p in params.items()}, cams, RasterConfig())
    ref = r.backward((torch.sign(im2 - t.reshape(-1)) / im2.numel()).contiguous())
    torch.cuda.synchronize()
    for k in PARAMS:
        assert params[k].grad.dtype == params[k].dtype
        e = rel_l2(params[k].grad.float().cpu().numpy(), ref[k].cpu().numpy())
        assert e <= (1e-2 if k in STORED else ATOMIC_TOL), (k, e)
