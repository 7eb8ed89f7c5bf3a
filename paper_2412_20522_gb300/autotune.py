"""Autotuner of the step's launch choices, and the CUDA-graph step runner.

Three choices change the speed of a masked forward+backward step but no
result the method defines (each is parity-tested against the oracle):

* the tile shape (16x16, 8x32 or 32x8; the image depends slightly on it
  through the 3-sigma tile rectangle, which is why every shape has its own
  oracle parity tests);
* the staging depth of the render kernels: splats staged in shared memory per
  batch, 256 or 128 in the forward, 128 or 64 in the backward;
* the digit width of the tile sort: the depth order of the records followed
  by a stable sort of the instances in 8-bit tile-id digits ("radix8"), or
  one counting pass over the whole tile id with each tile's list then put in
  depth order in shared memory ("bucket").

``autotune`` times a captured step for each choice (coordinate search: the
tile shape first, then the sort, then the staging depths, each with the
best so far) and caches the winner per (GPU, resolutions, Gaussian count,
storage) in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from .rasterize import PARAM_NAMES, RasterConfig, Rasterizer

TILE_SHAPES = ((16, 16), (8, 32), (32, 8))
SORTS = ("radix8", "bucket")
FWD_BATCHES = (256, 128)
BWD_BATCHES = (128, 64)


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
    then replays the whole sequence (no host synchronisation inside).

    A captured step keeps the arguments it was captured with, the mask
    sample's iteration among them.  With ``advance_iteration`` the iteration
    lives in a device counter (``self.iteration``: the next replay samples
    with cfg.iteration + its value) that the step itself advances by one
    after the backward, so successive replays draw successive Gumbel masks
    (Sec. 3.3), as a training loop needs.  The counter counts every step run,
    the warm-up ones included; set it (``self.iteration.fill_(k)``) to choose
    the next replay's iteration."""

    def __init__(self, params, cams, cfg: RasterConfig, target, view_ranges=None, warmup=2,
                 tile_order=True, advance_iteration=False, iteration=None):
        self.params = params
        self.cams = cams
        # ``iteration``: a device counter (int64 [1]) to read and advance,
        # shared with other captured steps (the slots of a pipeline, replayed
        # in turn on one stream); implies advance_iteration
        self.advance_iteration = advance_iteration or iteration is not None
        self.iteration = iteration
        if self.advance_iteration:
            import dataclasses
            if self.iteration is None:
                self.iteration = torch.zeros(1, dtype=torch.int64, device=params["means"].device)
            cfg = dataclasses.replace(cfg, iteration_dev=self.iteration)
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
        if self.advance_iteration:
            from . import abi
            abi.mg_advance_iteration(self.iteration, 1, self.rast._stream())
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


TUNED = ("tile_w", "tile_h", "sort", "render_batch", "render_batch_bwd")


def _load_cache(path):
    if os.path.exists(path):
        try:
            with open(path) as fh:
                return json.load(fh)
        except (OSError, ValueError):
            return {}
    return {}


def autotune(params, cams, target, base_cfg: RasterConfig | None = None, view_ranges=None,
             steps=5, use_cache=True) -> RasterConfig:
    """The fastest tile shape, sort digit width and staging depths for this
    workload (cached), as a RasterConfig built on ``base_cfg``."""
    base = base_cfg or RasterConfig()
    key = _key(params, cams)
    path = cache_path()
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache and all(k in cache[key] for k in TUNED):
        return RasterConfig(**{**base.__dict__, **{k: cache[key][k] for k in TUNED}})
    timings = {}

    def run(choice):
        name = "{tile_w}x{tile_h}|{sort}|{render_batch}/{render_batch_bwd}".format(**choice)
        if name not in timings:
            cfg = RasterConfig(**{**base.__dict__, **choice})
            gs = GraphStep(params, cams, cfg, target, view_ranges)
            timings[name] = time_step(gs.replay, steps=steps)
            del gs
            torch.cuda.empty_cache()
        return timings[name]

    best = dict(tile_w=base.tile_w, tile_h=base.tile_h, sort=base.sort,
                render_batch=base.render_batch or 256, render_batch_bwd=base.render_batch_bwd or 128)
    searches = ([dict(tile_w=w, tile_h=h) for w, h in TILE_SHAPES],
                [dict(sort=m) for m in SORTS],
                [dict(render_batch=b) for b in FWD_BATCHES],
                [dict(render_batch_bwd=b) for b in BWD_BATCHES])
    for options in searches:
        best = min(({**best, **o} for o in options), key=run)
    cache[key] = {**best, "ms": timings}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return RasterConfig(**{**base.__dict__, **best})


def autotune_tile(params, cams, target, base_cfg: RasterConfig | None = None, view_ranges=None,
                  steps=5, use_cache=True) -> tuple:
    """The tile shape of ``autotune``'s choice."""
    cfg = autotune(params, cams, target, base_cfg, view_ranges, steps, use_cache)
    return cfg.tile_w, cfg.tile_h
