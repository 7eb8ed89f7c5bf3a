"""Oracle: pruning of Sec. 3.5 (test infrastructure only).

Every Gaussian is sampled ``n_draws`` times (the paper: 10) and the ones never
sampled present are removed; the survivors keep their order.
"""
from __future__ import annotations

import numpy as np

from . import fp32_path

ATTRS = ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")


def keep_mask(mask_logits, seed, iteration, n_draws=10, index_offset=0):
    return fp32_path.prune_keep(mask_logits, seed, iteration, n_draws, index_offset)


def compact(arrays: dict, keep) -> tuple:
    """Rows with keep != 0 of every array, in order; new_index[i] = the row of
    i among the survivors, -1 if removed.  Returns (arrays, new_index, count)."""
    keep = np.asarray(keep).astype(bool)
    new_index = np.full(keep.shape[0], -1, np.int64)
    new_index[keep] = np.arange(int(keep.sum()))
    return {k: np.asarray(v)[keep] for k, v in arrays.items()}, new_index, int(keep.sum())
