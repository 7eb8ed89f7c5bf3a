"""Oracle: tile binning and depth ordering (test infrastructure only).

Sec. 3.1: only Gaussians intersecting a tile of the 16x16 grid take part in
that tile's pixels, and each pixel blends its Gaussians in depth order.
Instances are emitted per visible Gaussian in index order, tiles row-major
within its rectangle, with key (tile << 32) | depth_bits; the tile filter of
the decision path drops the pairs where the Gaussian stays under the alpha
floor in the whole tile; a stable sort by key orders each tile's list by
depth and breaks depth ties by Gaussian index.  numpy's stable argsort
serves as the sort primitive.
"""
from __future__ import annotations

import numpy as np

from . import fp32_path


def emit_instances(fp32, grid_w, tile_w=16, tile_h=16):
    """Keys (uint64) and values (uint32 Gaussian index) in emission order,
    the exclusive prefix sum of tiles-touched (uint64), K (the rectangle's
    instances) and keep (bool per instance): the decision-path tile filter
    (``fp32_path.tile_hit``) that drops the pairs where the Gaussian is under
    the alpha floor at every pixel of the tile."""
    tiles = fp32["tiles"].astype(np.int64)
    n = tiles.shape[0]
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(tiles, out=offsets[1:])
    K = int(offsets[-1])
    # instance k of Gaussian g covers tile (x0 + k % w, y0 + k // w), row-major
    g = np.repeat(np.arange(n, dtype=np.int64), tiles)
    local = np.arange(K, dtype=np.int64) - offsets[:-1][g]
    w = (fp32["x1"] - fp32["x0"] + 1).astype(np.int64)[g]
    tx = fp32["x0"].astype(np.int64)[g] + local % w
    ty = fp32["y0"].astype(np.int64)[g] + local // w
    tid = (ty * grid_w + tx).astype(np.uint64)
    keys = (tid << np.uint64(32)) | fp32["depth_bits"].astype(np.uint64)[g]
    vals = g.astype(np.uint32)
    tdet, rba, rbc = fp32_path.tile_filter_params(fp32)
    keep = fp32_path.tile_hit(fp32["px"][g], fp32["py"][g], fp32["a"][g], fp32["b"][g],
                              fp32["c"][g], tdet[g], rba[g], rbc[g], tx, ty, tile_w, tile_h)
    return keys, vals, offsets[:-1].astype(np.uint64), K, keep


def sort_instances(keys, vals):
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order]


def tile_ranges(sorted_keys, n_tiles):
    """ranges[t] = [start, end) of the instances whose key >> 32 == t."""
    tile = (sorted_keys >> np.uint64(32)).astype(np.int64)
    t = np.arange(n_tiles, dtype=np.int64)
    start = np.searchsorted(tile, t, side="left")
    end = np.searchsorted(tile, t, side="right")
    return np.stack([start, end], axis=1).astype(np.uint32)


def depth_order(depth_bits, visible):
    """Records ordered by the float bits of their depth (stable: ties keep
    record order), records outside every tile last."""
    keys = np.where(visible, depth_bits.astype(np.uint64), np.uint64(0xFFFFFFFF))
    return np.argsort(keys, kind="stable").astype(np.uint32)
