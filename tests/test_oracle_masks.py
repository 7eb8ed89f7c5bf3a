"""Pins of the oracle's mask loss (Sec. 3.5, Eq. 7-8), the ablations of
Sec. 4.3 (threshold mask with a straight-through sigmoid; mask multiplied
into the opacity) and the pruning rule of Sec. 3.5 -- each against something
other than the oracle's own formula: finite differences of a smooth
surrogate, the Gumbel-max theorem, the identity between the two ways of
removing a Gaussian from the blend, and plain loops."""
import math

import numpy as np
import pytest
import torch

from oracle import fp32_path as fp
from oracle import pipeline, preprocess, pruning
from paper_2412_20522_gb300 import scenes


def _scene(n=60, seed=11):
    g = scenes.uniform_gaussians(n, seed=seed, log_scale_mu=-2.6)
    cams = [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 32, 24, 30.0),
            scenes.look_at_camera((1.0, 0.3, -2.8), (0, 0, 0), 24, 32, 28.0)]
    return g, cams


def _zero_grads(cams):
    return [np.zeros((3, c.height, c.width)) for c in cams]


def test_mask_loss_value_closed_form():
    g, cams = _scene()
    given = (np.arange(g.n) % 4 == 0).astype(np.uint8)          # 15 of 60 present
    for kind, expect in ((pipeline.LOSS_L2, 0.25 ** 2), (pipeline.LOSS_L1, 0.25)):
        cfg = pipeline.OracleConfig(mask_mode=pipeline.MASK_GIVEN, given_mask=given,
                                    lambda_m=0.7, mask_loss=kind)
        assert pipeline.mask_loss(given, cfg) == pytest.approx(0.7 * expect, rel=1e-15)
    cfg = pipeline.OracleConfig(lambda_m=0.0)
    assert pipeline.mask_loss(given, cfg) == 0.0


@pytest.mark.parametrize("kind", [pipeline.LOSS_L2, pipeline.LOSS_L1])
@pytest.mark.parametrize("mode", [pipeline.MASK_GUMBEL, pipeline.MASK_STE])
def test_mask_loss_gradient_matches_fd_of_straight_through_surrogate(kind, mode):
    """With no render gradient, dL/dl is lambda_m dL_m/dl through the
    straight-through mask: the derivative of L_m(M + s(l) - s(l_ref)) with the
    hard sample held fixed, s the soft sample (Gumbel-softmax y_0 or the
    sigmoid).  Central differences of that smooth function pin it."""
    g, cams = _scene()
    lam = 0.37
    cfg = pipeline.OracleConfig(seed=5, iteration=3, lambda_m=lam, mask_loss=kind,
                                mask_mode=mode, ste_logit=-0.2, tau=0.8)
    views, M, minfo = pipeline.forward(g, cams, cfg)
    grads, _ = pipeline.backward(g, cams, cfg, views, M, minfo, _zero_grads(cams))
    l_ref = g.mask_logits.astype(np.float64)
    n = g.n

    def soft(l):
        if mode == pipeline.MASK_GUMBEL:
            g0 = -np.log(-np.log(minfo["u0"].astype(np.float64)))
            g1 = -np.log(-np.log(minfo["u1"].astype(np.float64)))
            z0, z1 = (l[:, 0] + g0) / cfg.tau, (l[:, 1] + g1) / cfg.tau
            return 1.0 / (1.0 + np.exp(z1 - z0))
        return 1.0 / (1.0 + np.exp(-(l[:, 0] - l[:, 1])))

    s_ref = soft(l_ref)

    def L(l):
        frac = (M + soft(l) - s_ref).sum() / n
        return lam * (frac * frac if kind == pipeline.LOSS_L2 else frac)

    rng = np.random.default_rng(3)
    for i in rng.choice(n, 15, replace=False):
        for k in (0, 1):
            h = 1e-5
            lp, lm = l_ref.copy(), l_ref.copy()
            lp[i, k] += h
            lm[i, k] -= h
            fd = (L(lp) - L(lm)) / (2 * h)
            assert fd == pytest.approx(grads["mask_logits"][i, k], rel=1e-6, abs=1e-13)
    # every other parameter is untouched by L_m
    for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert np.abs(grads[name]).max() == 0.0


def test_mask_loss_gradient_adds_to_render_gradient():
    g, cams = _scene()
    rng = np.random.default_rng(4)
    ws = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    base = dict(seed=5, iteration=3)
    cfg0 = pipeline.OracleConfig(**base)
    cfg1 = pipeline.OracleConfig(lambda_m=0.2, **base)
    views, M, minfo = pipeline.forward(g, cams, cfg0)
    g0, _ = pipeline.backward(g, cams, cfg0, views, M, minfo, ws)
    g1, _ = pipeline.backward(g, cams, cfg1, views, M, minfo, ws)
    gl, _ = pipeline.backward(g, cams, cfg1, views, M, minfo, _zero_grads(cams))
    assert np.allclose(g1["mask_logits"], g0["mask_logits"] + gl["mask_logits"], rtol=1e-12,
                       atol=1e-15)
    assert np.allclose(g1["means"], g0["means"], rtol=1e-12, atol=1e-15)


def test_ste_mask_is_sigmoid_threshold():
    rng = np.random.default_rng(5)
    l = rng.standard_normal((100_000, 2)).astype(np.float32) * 3
    theta = 0.01                                      # a threshold of the kind the ablation uses
    t32 = np.float32(math.log(theta / (1 - theta)))
    M, d = fp.ste_mask(l, t32)
    p = 1.0 / (1.0 + np.exp(-(l[:, 0].astype(np.float64) - l[:, 1])))
    clear = np.abs(p - theta) > 1e-6 * theta
    assert np.array_equal(M[clear].astype(bool), (p > theta)[clear])
    assert clear.mean() > 0.999
    # deterministic: no dependence on seed or iteration
    g, cams = _scene()
    cfg = pipeline.OracleConfig(mask_mode=pipeline.MASK_STE, ste_logit=float(t32))
    a = pipeline.sample_masks(g, cfg)[0]
    cfg.seed, cfg.iteration = 9, 99
    assert np.array_equal(a, pipeline.sample_masks(g, cfg)[0])


def test_opacity_ablation_against_masked_rasterisation():
    """Masking by opacity (o' = M o) and masked rasterisation remove a
    Gaussian from the blend in the same way (alpha 0 is filtered; M = 0 leaves
    T and C alone), so images and every gradient but the mask's agree.  The
    mask gradients differ exactly where the paper says (Sec. 4.3): zero for
    masked Gaussians under opacity masking, and for sampled ones
    o dL/do' = sum alpha dL/dalpha = Eq. 6 at M = 1 (no alpha at the 0.99 clamp
    here: every o < 0.99)."""
    g, cams = _scene()
    assert (g.opacity_logit < math.log(0.99 / 0.01)).all()
    rng = np.random.default_rng(6)
    ws = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    res = {}
    for apply in (pipeline.APPLY_RASTER, pipeline.APPLY_OPACITY):
        cfg = pipeline.OracleConfig(seed=5, iteration=3, bg=(0.2, 0.3, 0.1), mask_apply=apply)
        views, M, minfo = pipeline.forward(g, cams, cfg)
        grads, per_view = pipeline.backward(g, cams, cfg, views, M, minfo, ws)
        res[apply] = (views, M, grads)
    (vr, M, gr), (vo, Mo, go) = res[pipeline.APPLY_RASTER], res[pipeline.APPLY_OPACITY]
    assert np.array_equal(M, Mo)
    assert 0 < M.sum() < g.n
    for a, b in zip(vr, vo):
        assert np.array_equal(a.out["image"], b.out["image"])
        assert np.array_equal(a.out["final_T"], b.out["final_T"])
        assert np.array_equal(a.out["n_contrib"], b.out["n_contrib"])
    for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        assert np.allclose(go[name], gr[name], rtol=1e-10, atol=1e-14), name
    off = M == 0
    assert np.abs(go["mask_logits"][off]).max() == 0.0
    assert np.abs(gr["mask_logits"][off]).max() > 0.0          # masked rasterisation reaches them
    assert np.allclose(go["mask_logits"][~off], gr["mask_logits"][~off], rtol=1e-9, atol=1e-15)


def test_prune_keep_frequency():
    """Gumbel-max theorem per draw: P(never sampled in n draws) = (1 - p)^n
    with p = sigmoid(l_0 - l_1) (Sec. 3.5)."""
    n = 100_000
    for l0, l1, draws in [(0.0, 0.0, 10), (-3.0, 0.0, 10), (-5.0, 0.5, 10), (-1.0, 0.0, 3)]:
        logits = np.tile(np.array([[l0, l1]], np.float32), (n, 1))
        keep = fp.prune_keep(logits, seed=42, it=7, n_draws=draws)
        p = 1.0 / (1.0 + math.exp(-(l0 - l1)))
        q = 1.0 - (1.0 - p) ** draws
        sd = math.sqrt(q * (1 - q) / n)
        assert abs(keep.mean() - q) < 5 * sd + 1e-12, (l0, l1, keep.mean(), q)


def test_prune_draws_are_not_the_training_draw_and_nest():
    l = np.zeros((50_000, 2), np.float32)
    train = fp.sample_mask(l, 3, 11)[0].astype(float)
    one = fp.prune_keep(l, 3, 11, n_draws=1)
    assert np.array_equal(one, fp.sample_mask(l, 3, 11, draw=1)[0])
    assert abs(np.corrcoef(train, one.astype(float))[0, 1]) < 0.03
    k5 = fp.prune_keep(l, 3, 11, n_draws=5)
    k10 = fp.prune_keep(l, 3, 11, n_draws=10)
    assert (k10 >= k5).all() and (k5 >= one).all()


def test_compact_matches_loop():
    rng = np.random.default_rng(7)
    n = 257
    arrays = {"means": rng.standard_normal((n, 3)), "sh": rng.standard_normal((n, 16, 3)),
              "opacity_logit": rng.standard_normal(n)}
    keep = (rng.random(n) < 0.4).astype(np.uint8)
    out, new_index, count = pruning.compact(arrays, keep)
    rows = [i for i in range(n) if keep[i]]
    assert count == len(rows)
    for k, v in arrays.items():
        assert np.array_equal(out[k], np.stack([v[i] for i in rows]))
    for j, i in enumerate(rows):
        assert new_index[i] == j
    assert (new_index[keep == 0] == -1).all()
    empty, ni, c = pruning.compact(arrays, np.zeros(n, np.uint8))
    assert c == 0 and empty["sh"].shape == (0, 16, 3) and (ni == -1).all()
