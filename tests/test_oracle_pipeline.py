"""End-to-end pins of the oracle's forward+backward: parameter gradients
against central finite differences of the FP64 forward (with the discrete
structure -- visibility, tile lists, depth order, hard mask -- held fixed),
and the straight-through mask gradient against finite differences of the
soft Gumbel-softmax sample (Sec. 3.3)."""
import numpy as np
import pytest
import torch

from oracle import pipeline, preprocess, render
from paper_2412_20522_gb300 import scenes


def _scene(bg=(0.3, 0.1, 0.6)):
    g = scenes.uniform_gaussians(60, seed=11, log_scale_mu=-2.6)
    cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 32, 24, 30.0),
            scenes.look_at_camera((1.0, 0.3, -2.8), (0, 0, 0), 24, 32, 28.0)]
    cfg = pipeline.OracleConfig(bg=bg, seed=5, iteration=3)
    return g, cams, cfg


def _images(p64, cams, views, M, cfg):
    """FP64 forward with the discrete structure of ``views`` held fixed."""
    imgs = []
    for cam, v in zip(cams, views):
        vis = v.visible
        with torch.no_grad():
            sp = preprocess.splat({k: t[vis] for k, t in p64.items()}, cam)
        n = M.shape[0]
        mean2d = np.zeros((n, 2)); conic = np.zeros((n, 3)); op = np.zeros(n); rgb = np.zeros((n, 3))
        mean2d[vis] = sp["mean2d"].numpy(); conic[vis] = sp["conic"].numpy()
        op[vis] = sp["opacity"].numpy(); rgb[vis] = sp["rgb"].numpy()
        s = render.SplatsF64(mean2d, conic, op, rgb, M.astype(np.float64))
        imgs.append(render.render_tiled(s, cam.width, cam.height, cfg.tile_w, cfg.tile_h,
                                        v.sorted_vals, v.ranges, cfg.bg, 1))
    return imgs


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.1, 0.6)])
def test_parameter_gradients_match_finite_differences(bg):
    g, cams, cfg = _scene(bg)
    views, M, minfo = pipeline.forward(g, cams, cfg)
    rng = np.random.default_rng(2)
    ws = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    grads, _ = pipeline.backward(g, cams, cfg, views, M, minfo, ws)
    base = pipeline.gaussian_params64(g)
    ref = _images(base, cams, views, M, cfg)
    seen = set()
    for v in views:
        seen |= set(v.visible.tolist())
    checked = {}
    for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        arr = base[name]
        per = arr[0].numel()
        cand = [i for i in range(arr.numel()) if i // per in seen]
        for i in rng.choice(cand, 25, replace=False):
            h = 1e-6 * max(1.0, abs(float(arr.reshape(-1)[i])))
            Ls = []
            ok = True
            for sgn in (1, -1):
                p = {k: t.clone() for k, t in base.items()}
                p[name].reshape(-1)[i] += sgn * h
                imgs = _images(p, cams, views, M, cfg)
                if any(not np.array_equal(a["n_contrib"], b["n_contrib"]) for a, b in zip(imgs, ref)):
                    ok = False
                Ls.append(sum(float((im["image"] * w).sum()) for im, w in zip(imgs, ws)))
            if not ok:
                continue
            fd = (Ls[0] - Ls[1]) / (2 * h)
            an = float(grads[name].reshape(-1)[i])
            assert fd == pytest.approx(an, rel=2e-4, abs=1e-7), (name, i, fd, an)
            checked[name] = checked.get(name, 0) + 1
    assert all(checked.get(n, 0) >= 15 for n in ("means", "log_scales", "quats",
                                                 "opacity_logit", "sh")), checked


def test_straight_through_mask_gradient_is_soft_sample_derivative():
    g, cams, cfg = _scene()
    views, M, minfo = pipeline.forward(g, cams, cfg)
    rng = np.random.default_rng(6)
    ws = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    grads, _ = pipeline.backward(g, cams, cfg, views, M, minfo, ws)
    dM = grads["dmask"]
    logits = torch.as_tensor(g.mask_logits.astype(np.float64))

    def soft(l):
        return float((preprocess.mask_straight_through(l, M, minfo["u0"], minfo["u1"],
                                                       cfg.tau)[1].numpy() * dM).sum())
    for i in rng.choice(g.n, 20, replace=False):
        for k in (0, 1):
            h = 1e-6
            lp, lm = logits.clone(), logits.clone()
            lp[i, k] += h
            lm[i, k] -= h
            fd = (soft(lp) - soft(lm)) / (2 * h)
            assert fd == pytest.approx(grads["mask_logits"][i, k], rel=1e-5, abs=1e-12)
    # two-category softmax: the two logits' gradients are opposite
    assert np.allclose(grads["mask_logits"][:, 0], -grads["mask_logits"][:, 1])
    assert np.count_nonzero(grads["mask_logits"]) > 0


def test_mask_gradient_is_exact_derivative_of_blend():
    """dL/dM_i summed over views equals the FD of the image w.r.t. M_i, for
    masked and unmasked Gaussians alike (the point of masked rasterisation)."""
    g, cams, cfg = _scene()
    views, M, minfo = pipeline.forward(g, cams, cfg)
    rng = np.random.default_rng(8)
    ws = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    grads, _ = pipeline.backward(g, cams, cfg, views, M, minfo, ws)
    p = pipeline.gaussian_params64(g)
    n_checked = [0, 0]
    ref = _images(p, cams, views, M.astype(np.float64), cfg)
    h = 1e-3
    for i in rng.choice(g.n, 30, replace=False):
        Ls = []
        same = True
        for d in (h, -h):
            Mp = M.astype(np.float64).copy()
            Mp[i] += d
            imgs = _images(p, cams, views, Mp, cfg)
            same &= all(np.array_equal(a["n_contrib"], b["n_contrib"]) for a, b in zip(imgs, ref))
            Ls.append(sum(float((im["image"] * w).sum()) for im, w in zip(imgs, ws)))
        fd = (Ls[0] - Ls[1]) / (2 * h)
        if same and (abs(grads["dmask"][i]) > 0 or abs(fd) > 0):
            assert fd == pytest.approx(grads["dmask"][i], rel=1e-8, abs=1e-11)
            n_checked[int(M[i])] += 1
    assert min(n_checked) >= 3
