"""Oracle: one masked forward + backward of MaskGaussian (test infrastructure only).

Forward (Sec. 3.2-3.3, Fig. 2): sample the masks, splat every Gaussian with no
attribute masked, bin into tiles, depth-order, composite with Eq. 3-4.
Loss: L1 between the rendered and a target image, mean over 3 H W
(``L_render``; the paper does not state its form, an L1 reading), per view,
summed over views.  Backward: Eq. 6 + Appendix A for the mask, the colour and
alpha gradients of the same blend, then the exact derivative of the splat
(autograd in FP64) down to the Gaussian parameters and, through the
Gumbel-softmax straight-through estimator, to the two existence scores.
The mask loss of Eq. 7-8 (lambda_m L_m) is added to the loss and its
gradient flows through the same straight-through mask.  Ablations of
Sec. 4.3: the deterministic threshold mask with a sigmoid straight-through
gradient, and the mask multiplied into the opacity instead of masked
rasterisation.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import binning, fp32_path, preprocess, render

MASK_GUMBEL, MASK_ALL_ONES, MASK_GIVEN, MASK_STE = 0, 1, 2, 3
APPLY_RASTER, APPLY_OPACITY = 0, 1
LOSS_L2, LOSS_L1 = 0, 1
PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")


@dataclass
class OracleConfig:
    tile_w: int = 16
    tile_h: int = 16
    bg: tuple = (0.0, 0.0, 0.0)
    seed: int = 2024124
    iteration: int = 0
    tau: float = 1.0
    mask_mode: int = MASK_GUMBEL
    given_mask: np.ndarray | None = None
    eps: float = 1e-3           # straddle band of the alpha floor / power sign (relative)
    eps_T: float = 1e-3         # straddle band of the termination test (relative)
    index_offset: int = 0       # index of the first Gaussian in a batch of scenes (noise counter)
    mask_apply: int = APPLY_RASTER   # masked rasterisation (Eq. 3-4) or mask x opacity (Sec. 4.3)
    lambda_m: float = 0.0       # weight of the mask loss, Eq. 8
    mask_loss: int = LOSS_L2    # Eq. 7 (squared mean) or the L1 form of Appendix C
    ste_logit: float = 0.0      # MASK_STE threshold on l_0 - l_1 (FP32)
    bin_mode: int = 0           # 0: tile-filtered lists; 1: whole 3-sigma rectangles


@dataclass
class OracleView:
    fp32: dict
    keys: np.ndarray
    vals: np.ndarray
    offsets: np.ndarray
    K: int
    sorted_keys: np.ndarray
    sorted_vals: np.ndarray
    ranges: np.ndarray
    visible: np.ndarray
    splats: render.SplatsF64
    out: dict
    values64: dict = field(default_factory=dict)
    keep: np.ndarray | None = None     # tile filter per emitted instance

    @property
    def K_kept(self) -> int:
        """Instances in the tile lists (the rectangle's K minus the filtered)."""
        return int(self.sorted_vals.shape[0])


def gaussian_params64(g) -> dict:
    return {name: torch.as_tensor(np.asarray(getattr(g, name), dtype=np.float64))
            for name in PARAM_NAMES}


def sample_masks(g, cfg: OracleConfig):
    n = g.n
    if cfg.mask_mode == MASK_ALL_ONES:
        return np.ones(n, np.uint8), None
    if cfg.mask_mode == MASK_GIVEN:
        return np.asarray(cfg.given_mask, dtype=np.uint8).copy(), None
    if cfg.mask_mode == MASK_STE:
        M, d = fp32_path.ste_mask(g.mask_logits, cfg.ste_logit)
        return M, dict(margin=d)
    M, margin, u0, u1 = fp32_path.sample_mask(g.mask_logits, cfg.seed, cfg.iteration,
                                              cfg.index_offset)
    return M, dict(margin=margin, u0=u0, u1=u1)


def mask_loss(M, cfg: OracleConfig) -> float:
    """lambda_m L_m of Eq. 7-8 (L2: the squared fraction of present Gaussians;
    L1: the fraction itself), over the N Gaussians of the scene."""
    n = len(M)
    if n == 0 or cfg.lambda_m == 0.0:
        return 0.0
    frac = float(np.sum(np.asarray(M, np.float64))) / n
    return cfg.lambda_m * (frac * frac if cfg.mask_loss == LOSS_L2 else frac)


def _mask_st(p64, M, minfo, cfg: OracleConfig):
    """The mask as a differentiable tensor: hard value, straight-through
    gradient (Sec. 3.3 for Gumbel-softmax, the sigmoid for the threshold
    ablation); a constant for all-ones and given masks."""
    if cfg.mask_mode == MASK_GUMBEL:
        return preprocess.mask_straight_through(p64["mask_logits"], M, minfo["u0"], minfo["u1"],
                                                cfg.tau)[0]
    if cfg.mask_mode == MASK_STE:
        return preprocess.mask_straight_through_ste(p64["mask_logits"], M)[0]
    return torch.as_tensor(np.asarray(M, np.float64))


def forward(g, cams, cfg: OracleConfig):
    """Masked forward over all cameras. Returns (views, mask, mask_info)."""
    M, minfo = sample_masks(g, cfg)
    p64 = gaussian_params64(g)
    views = []
    for cam in cams:
        fp = fp32_path.project32(g.means, g.log_scales, g.quats, cam, cfg.tile_w, cfg.tile_h)
        gx, gy = fp["grid"]
        # the binning's candidates: the whole 3-sigma rectangle, or (tile
        # filter) its tiles that the filter can keep; the square stays in
        # rect_tiles
        fp["rect_tiles"] = fp["tiles"]
        if cfg.bin_mode == 0:
            fp.update(fp32_path.candidate_rect(fp, cfg.tile_w, cfg.tile_h))
        keys, vals, offsets, K, keep = binning.emit_instances(fp, gx, cfg.tile_w, cfg.tile_h)
        if cfg.bin_mode == 1:
            keep = np.ones_like(keep)
        skeys, svals = binning.sort_instances(keys[keep], vals[keep])
        ranges = binning.tile_ranges(skeys, gx * gy)
        vis = np.nonzero(fp["visible"])[0]
        n = g.n
        mean2d = np.zeros((n, 2))
        conic = np.zeros((n, 3))
        opac = np.zeros(n)
        rgb = np.zeros((n, 3))
        with torch.no_grad():
            sub = {k: v[vis] for k, v in p64.items()}
            sp = preprocess.splat(sub, cam)
        mean2d[vis] = sp["mean2d"].numpy()
        conic[vis] = sp["conic"].numpy()
        opac[vis] = sp["opacity"].numpy()
        rgb[vis] = sp["rgb"].numpy()
        if cfg.mask_apply == APPLY_OPACITY:
            # ablation: the mask scales the opacity, every splat blends unmasked
            splats = render.SplatsF64(mean2d, conic, opac * M, rgb, np.ones(n))
        else:
            splats = render.SplatsF64(mean2d, conic, opac, rgb, M.astype(np.float64))
        out = render.render_tiled(splats, cam.width, cam.height, cfg.tile_w, cfg.tile_h,
                                  svals, ranges, cfg.bg, True, cfg.eps, cfg.eps_T)
        views.append(OracleView(fp, keys, vals, offsets, K, skeys, svals, ranges, vis,
                                splats, out,
                                dict(mean2d=mean2d, conic=conic, opacity=opac, rgb=rgb,
                                     rgb_clamped=np.zeros((n, 3), bool)), keep))
        views[-1].values64["rgb_clamped"][vis] = sp["rgb_clamped"].numpy()
    return views, M, minfo


def l1_loss_grad(image, target):
    """L = mean |C - target| over 3 H W; dL/dC = sign(C - target) / (3 H W)."""
    diff = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return float(np.abs(diff).mean()), np.sign(diff) / diff.size


def backward(g, cams, cfg: OracleConfig, views, M, minfo, dL_dimages):
    """Gradients of sum_v <dL_dimages[v], image_v> w.r.t. every parameter.

    Returns (param_grads dict of float64 arrays, per_view render grads list).
    """
    per_view = []
    dmask_total = np.zeros(g.n)
    for cam, v, gimg in zip(cams, views, dL_dimages):
        rg = render.render_backward(v.splats, cam.width, cam.height, cfg.tile_w, cfg.tile_h,
                                    v.sorted_vals, v.ranges, gimg, cfg.bg)
        per_view.append(rg)
        dmask_total += rg["dmask"]

    p64 = {k: t.clone().requires_grad_(True) for k, t in gaussian_params64(g).items()}
    Mst = _mask_st(p64, M, minfo, cfg)
    total = torch.zeros((), dtype=torch.float64)
    for cam, v, rg in zip(cams, views, per_view):
        vis = torch.as_tensor(v.visible)
        sub = {k: t[vis] for k, t in p64.items()}
        sp = preprocess.splat(sub, cam)
        idx = v.visible
        opacity = sp["opacity"]
        if cfg.mask_apply == APPLY_OPACITY:
            opacity = opacity * Mst[vis]          # o' = M o
        total = total + (sp["mean2d"] * torch.as_tensor(rg["dmean2d"][idx])).sum()
        total = total + (sp["conic"] * torch.as_tensor(rg["dconic"][idx])).sum()
        total = total + (opacity * torch.as_tensor(rg["dopacity"][idx])).sum()
        total = total + (sp["rgb"] * torch.as_tensor(rg["drgb"][idx])).sum()
    if cfg.mask_apply == APPLY_RASTER:
        total = total + (Mst * torch.as_tensor(dmask_total)).sum()
    if cfg.lambda_m != 0.0 and g.n > 0:
        frac = Mst.sum() / g.n
        total = total + cfg.lambda_m * (frac * frac if cfg.mask_loss == LOSS_L2 else frac)
    if total.requires_grad:
        total.backward()
    grads = {k: (t.grad.numpy() if t.grad is not None else np.zeros(tuple(t.shape)))
             for k, t in p64.items()}
    grads["dmask"] = dmask_total
    return grads, per_view


def forward_backward_l1(g, cams, targets, cfg: OracleConfig):
    views, M, minfo = forward(g, cams, cfg)
    loss = 0.0
    dimgs = []
    for v, tgt in zip(views, targets):
        l, d = l1_loss_grad(v.out["image"], tgt)
        loss += l
        dimgs.append(d)
    loss += mask_loss(M, cfg)
    grads, per_view = backward(g, cams, cfg, views, M, minfo, dimgs)
    return dict(views=views, mask=M, mask_info=minfo, loss=loss, dL_dimages=dimgs,
                grads=grads, per_view=per_view)
