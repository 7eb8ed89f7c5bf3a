"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

PARAMS = ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")


def to_device(g, device="cuda"):
    return {k: torch.as_tensor(np.ascontiguousarray(getattr(g, k))).to(device) for k in PARAMS}


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


def split_views(flat, cams, per_pixel_channels=3):
    out, o = [], 0
    for c in cams:
        n = per_pixel_channels * c.width * c.height
        shape = (per_pixel_channels, c.height, c.width) if per_pixel_channels > 1 else (c.height, c.width)
        out.append(flat[o:o + n].reshape(shape))
        o += n
    return out
