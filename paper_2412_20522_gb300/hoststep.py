"""Masked training steps on host-resident data, with the copies overlapped.

Every step copies its inputs (the Gaussian parameters and the target images)
from pinned host memory to the GPU and its results (image, loss and every
parameter gradient) back to pinned host memory.  The steps are pipelined
over three CUDA streams: the inputs of step i+1 travel while step i computes,
and the gradients of step i travel back while step i+1 computes.  Device
input and output buffers are double-buffered; events order every reuse.
All compute is the libmaskgs step: by default each slot replays its own
captured CUDA graph of the whole step (``autotune.GraphStep``, no launch
gaps); ``graph=False`` issues the same kernels one by one (``Rasterizer``).
With ``advance_iteration`` the steps share one device-side iteration counter
(``self.iteration``, mg_raster_cfg.iteration_dev) that each step advances
after its backward, so step k draws the Gumbel mask of iteration
cfg.iteration + k (Sec. 3.3); the counter starts at 0 for the first step.
"""
from __future__ import annotations

import torch

from .rasterize import PARAM_NAMES, RasterConfig, Rasterizer


class HostPipeline:
    def __init__(self, host_params: dict, host_target: torch.Tensor, cams, cfg: RasterConfig,
                 device="cuda", view_ranges=None, graph: bool = True,
                 advance_iteration: bool = False):
        self.dev = torch.device(device)
        self.iteration = None
        if advance_iteration:
            import dataclasses
            self.iteration = torch.zeros(1, dtype=torch.int64, device=self.dev)
            cfg = dataclasses.replace(cfg, iteration_dev=self.iteration)
        self.cams, self.cfg, self.view_ranges = cams, cfg, view_ranges
        for k, t in host_params.items():
            if not t.is_pinned():
                raise ValueError(f"{k}: pinned host memory required")
        self.host_params = host_params
        self.host_target = host_target
        self.params = [{k: torch.empty_like(v, device=self.dev) for k, v in host_params.items()}
                       for _ in range(2)]
        self.target = [torch.empty_like(host_target, device=self.dev) for _ in range(2)]
        self.grads = [{k: torch.empty(v.shape, dtype=torch.float32, device=self.dev)
                       for k, v in host_params.items()} for _ in range(2)]
        npix = 3 * sum(int(c.width) * int(c.height) for c in cams)
        # per-slot copies of the rasteriser's (single) image and loss buffers,
        # so that the next step may overwrite those while these travel
        self.image = [torch.empty(npix, dtype=torch.float32, device=self.dev) for _ in range(2)]
        self.loss = [torch.empty(1, dtype=torch.float32, device=self.dev) for _ in range(2)]
        self.h2d = torch.cuda.Stream(self.dev)
        self.d2h = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.Stream(self.dev)
        self.rast = Rasterizer(self.dev)
        self.host_grads = [{k: torch.empty(v.shape, dtype=torch.float32).pin_memory()
                            for k, v in host_params.items()} for _ in range(2)]
        self.host_image = [torch.empty(npix, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.host_loss = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.ev_in = [None, None]       # inputs of slot b on the device
        self.ev_comp = [None, None]     # step of slot b computed (inputs free, outputs ready)
        self.ev_out = [None, None]      # outputs of slot b on the host (device outputs free)
        # both slots' inputs, then (eager form) size the instance buffers once
        # with a synchronising forward; each GraphStep sizes its own
        with torch.cuda.stream(self.compute):
            for b in range(2):
                for k in PARAM_NAMES:
                    self.params[b][k].copy_(host_params[k])
                self.target[b].copy_(host_target)
            if not graph:
                self.rast.forward(self.params[0], cams, cfg, view_ranges=view_ranges, check=True)
        torch.cuda.synchronize(self.dev)
        self.graphs = None
        if graph:
            # one captured step per slot, reading that slot's inputs and
            # writing its own gradients, image and loss
            from .autotune import GraphStep
            self.graphs = [GraphStep(self.params[b], cams, cfg, self.target[b],
                                     view_ranges=view_ranges, iteration=self.iteration)
                           for b in range(2)]
            for b in range(2):
                self.grads[b] = self.graphs[b].grads
                self.image[b] = self.graphs[b].image
                self.loss[b] = self.graphs[b].loss
            torch.cuda.synchronize(self.dev)
        if self.iteration is not None:     # the warm-up steps advanced it: step 0 reads 0
            self.iteration.zero_()
            torch.cuda.synchronize(self.dev)
        self.i = 0

    def h2d_bytes(self) -> int:
        return sum(v.numel() * v.element_size() for v in self.host_params.values()) + \
            self.host_target.numel() * self.host_target.element_size()

    def d2h_bytes(self) -> int:
        return (sum(v.numel() * 4 for v in self.host_grads[0].values()) +
                self.host_image[0].numel() * 4 + 4)

    def step(self):
        """Enqueue one step (no host synchronisation)."""
        b = self.i & 1
        # inputs: wait until the step that last used this slot has computed
        with torch.cuda.stream(self.h2d):
            if self.ev_comp[b] is not None:
                self.h2d.wait_event(self.ev_comp[b])
            for k in PARAM_NAMES:
                self.params[b][k].copy_(self.host_params[k], non_blocking=True)
            self.target[b].copy_(self.host_target, non_blocking=True)
            self.ev_in[b] = torch.cuda.Event()
            self.ev_in[b].record(self.h2d)
        # compute: after the inputs arrived and the slot's previous outputs left
        with torch.cuda.stream(self.compute):
            self.compute.wait_event(self.ev_in[b])
            if self.ev_out[b] is not None:
                self.compute.wait_event(self.ev_out[b])
            if self.graphs is not None:
                self.graphs[b].replay()
            else:
                img, loss, dimg = self.rast.forward_l1(self.params[b], self.cams, self.cfg,
                                                       self.target[b],
                                                       view_ranges=self.view_ranges, check=False)
                self.rast.backward(dimg, self.grads[b])
                if self.iteration is not None:
                    from . import abi
                    abi.mg_advance_iteration(self.iteration, 1, self.rast._stream())
                self.image[b].copy_(img)
                self.loss[b].copy_(loss)
            self.ev_comp[b] = torch.cuda.Event()
            self.ev_comp[b].record(self.compute)
        # outputs back to the host
        with torch.cuda.stream(self.d2h):
            self.d2h.wait_event(self.ev_comp[b])
            self.host_image[b].copy_(self.image[b], non_blocking=True)
            self.host_loss[b].copy_(self.loss[b], non_blocking=True)
            for k in PARAM_NAMES:
                self.host_grads[b][k].copy_(self.grads[b][k], non_blocking=True)
            self.ev_out[b] = torch.cuda.Event()
            self.ev_out[b].record(self.d2h)
        self.i += 1
        return b

    def results(self, b):
        """Host image, loss and gradients of slot b (after synchronising)."""
        self.ev_out[b].synchronize()
        return self.host_image[b], self.host_loss[b], self.host_grads[b]
