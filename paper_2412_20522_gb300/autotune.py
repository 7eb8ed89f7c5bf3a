"""Tile-shape autotuner and CUDA-graph step runner.

The tile rectangle (and so the image) depends slightly on the tile shape,
which is why every shape is parity-tested against the oracle (tests run all
of 16x16, 8x32 and 32x8).  The autotuner times a full masked forward+backward
step for each shape and remembers the fastest per (GPU, resolution set,
Gaussian count) in a JSON cache file.  The staging depth (256 splats per
batch), the pixels per thread (2) and the sort digit width (8 bits) are
compile-time constants of libmaskgs, chosen by measurement.
"""
from __future__ import annotations

import json
import os

import torch

from .rasterize import PARAM_NAMES, RasterConfig, Rasterizer

TILE_SHAPES = ((16, 16), (8, 32), (32, 8))


def cache_path() -> str:
    return os.environ.get("MASKGS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "maskgs",
                                       "autotune.json"))


def _key(params, cams) -> str:
    dev = torch.cuda.get_device_name(params["means"].device)
    res = "+".join(f"{c.width}x{c.height}" for c in cams)
    return f"{dev}|{res}|n={int(params['means'].shape[0])}|{params['sh'].dtype}"


class GraphStep:
    """One masked forward + L1 loss + backward captured in a CUDA graph.

    All buffers are sized by a synchronising first step; the captured graph
    then replays the whole sequence (no host synchronisation inside)."""

    def __init__(self, params, cams, cfg: RasterConfig, target, view_ranges=None, warmup=2,
                 tile_order=True):
        self.params = params
        self.cams = cams
        self.cfg = cfg
        self.target = target
        self.view_ranges = view_ranges
        self.rast = Rasterizer(params["means"].device, tile_order=tile_order)
        self.grads = {k: torch.empty(params[k].shape, dtype=torch.float32,
                                     device=params[k].device) for k in PARAM_NAMES}
        self.rast.forward(params, cams, cfg, view_ranges=view_ranges, check=True)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self._step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.loss = self._step()

    def _step(self):
        img, loss, dimg = self.rast.forward_l1(self.params, self.cams, self.cfg, self.target,
                                               view_ranges=self.view_ranges, check=False)
        self.rast.backward(dimg, self.grads)
        self.image = img
        return loss

    def replay(self):
        self.graph.replay()

    def status(self):
        from . import abi
        return abi.mg_read_status(self.rast.status, self.rast._stream()).status


def time_step(fn, steps=5, warmup=2) -> float:
    """Mean ms of fn() over `steps`, CUDA events on the current stream."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def autotune_tile(params, cams, target, base_cfg: RasterConfig | None = None, view_ranges=None,
                  steps=5, use_cache=True) -> tuple:
    """Fastest tile shape for this workload (cached)."""
    key = _key(params, cams)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return tuple(cache[key]["tile"])
    base = base_cfg or RasterConfig()
    timings = {}
    for tw, th in TILE_SHAPES:
        cfg = RasterConfig(**{**base.__dict__, "tile_w": tw, "tile_h": th})
        gs = GraphStep(params, cams, cfg, target, view_ranges)
        timings[(tw, th)] = time_step(gs.replay, steps=steps)
        del gs
        torch.cuda.empty_cache()
    best = min(timings, key=timings.get)
    cache[key] = {"tile": list(best), "ms": {f"{a}x{b}": v for (a, b), v in timings.items()}}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as fh:
            json.dump(cache, fh, indent=1)
    except OSError:
        pass
    return best
