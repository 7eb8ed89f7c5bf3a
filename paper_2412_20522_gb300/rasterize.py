"""Masked rasterisation step on the GPU: buffers, launch sequence, autograd.

PyTorch provides device memory and the stream; every stage of the step runs
in libmaskgs through the C ABI (``abi``).  The per-step state kept between
forward and backward is per-pixel only (final transmittance and stop index):
the backward recomputes every fragment instead of storing it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import torch

from . import abi

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logit", "sh", "mask_logits")


@dataclass
class RasterConfig:
    tile_w: int = 16
    tile_h: int = 16
    bg: tuple = (0.0, 0.0, 0.0)
    tau: float = 1.0
    seed: int = 2024124
    iteration: int = 0
    mask_mode: int = abi.MG_MASK_GUMBEL
    given_mask: torch.Tensor | None = None     # uint8 [n] on the device
    mask_apply: int = abi.MG_APPLY_RASTER      # or MG_APPLY_OPACITY (ablation, Sec. 4.3)
    lambda_m: float = 0.0                      # mask-loss weight, Eq. 8
    mask_loss: int = abi.MG_MASK_LOSS_L2       # Eq. 7, or the L1 form
    ste_logit: float = 0.0                     # MG_MASK_STE threshold on l_0 - l_1
    bin_mode: int = abi.MG_BIN_FILTERED        # or MG_BIN_RECT (whole 3-sigma rectangles)
    # tile lists: "bucket" = one counting pass over the whole tile id and a
    # per-tile depth sort (mg_sort_by_tile); "radix8" = depth order of the
    # records, then a stable sort by tile id in 8-bit digits (mg_sort)
    sort: str = "radix8"
    # splats staged per batch by the render kernels (0 = the defaults: 256
    # forward, 128 backward; also 128 forward, 64 backward)
    render_batch: int = 0
    render_batch_bwd: int = 0
    # int64 [1] on the device (optional): added to `iteration` by the mask
    # sample, so a captured step draws a new mask each replay when the
    # counter is advanced between replays (abi.mg_advance_iteration)
    iteration_dev: torch.Tensor | None = None

    @staticmethod
    def ste_logit_of(theta: float) -> float:
        """The l_0 - l_1 threshold (an FP32 value) equivalent to
        sigmoid(l_0 - l_1) > theta."""
        import numpy as np
        return float(np.float32(math.log(theta / (1.0 - theta))))

    def c(self) -> abi.mg_raster_cfg:
        cfg = abi.mg_raster_cfg()
        cfg.tile_w, cfg.tile_h = self.tile_w, self.tile_h
        for i in range(3):
            cfg.bg[i] = float(self.bg[i])
        cfg.tau = float(self.tau)
        cfg.seed = int(self.seed)
        cfg.iteration = int(self.iteration)
        cfg.mask_mode = int(self.mask_mode)
        cfg.given_mask = abi.ptr(self.given_mask) if self.given_mask is not None else None
        cfg.mask_apply = int(self.mask_apply)
        cfg.lambda_m = float(self.lambda_m)
        cfg.mask_loss = int(self.mask_loss)
        cfg.ste_logit = float(self.ste_logit)
        cfg.bin_mode = int(self.bin_mode)
        cfg.render_batch = int(self.render_batch)
        cfg.render_batch_bwd = int(self.render_batch_bwd)
        cfg.iteration_dev = abi.ptr(self.iteration_dev) if self.iteration_dev is not None else None
        return cfg


def make_views(cams, ranges=None):
    """ctypes array of mg_view.  ``ranges``: per view (gaussian_offset, count);
    None means every view sees the same n Gaussians (set later by the caller)."""
    n = len(cams)
    if not 1 <= n <= abi.MG_MAX_VIEWS:
        raise ValueError(f"1..{abi.MG_MAX_VIEWS} views supported, got {n}")
    arr = (abi.mg_view * n)()
    for i, cam in enumerate(cams):
        c = arr[i].cam
        c.width, c.height = int(cam.width), int(cam.height)
        c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
        vm = [float(x) for x in cam.viewmat.reshape(-1)]
        for k in range(12):
            c.viewmat[k] = vm[k]
        for k in range(3):
            c.cam_pos[k] = float(cam.cam_pos[k])
        c.near_plane = float(cam.near)
        if ranges is not None:
            arr[i].gaussian_offset, arr[i].gaussian_count = (int(x) for x in ranges[i])
    return arr


_STORAGE = {torch.float32: abi.MG_DTYPE_F32, torch.bfloat16: abi.MG_DTYPE_BF16,
            torch.float16: abi.MG_DTYPE_F16}
STORED = ("log_scales", "quats", "opacity_logit", "sh")


def _gaussians_struct(p: dict, sh_degree: int) -> abi.mg_gaussians:
    """Means and mask logits are FP32; log-scales, quaternions, opacity logits
    and SH share one storage type (FP32, BF16 or FP16)."""
    g = abi.mg_gaussians()
    g.n = int(p["means"].shape[0])
    g.sh_degree = int(sh_degree)
    st = p["sh"].dtype
    if st not in _STORAGE:
        raise ValueError(f"unsupported attribute storage {st}")
    g.dtype = _STORAGE[st]
    for name in PARAM_NAMES:
        t = p[name]
        want = st if name in STORED else torch.float32
        if t.dtype != want or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name}: contiguous {want} CUDA tensor required")
        setattr(g, name, t.data_ptr())
    return g


class _Events:
    """Optional per-stage CUDA events {name: (start, end)} on the current
    stream, and optional NVTX ranges named after the stages (for a profiler's
    timeline)."""

    def __init__(self, events, nvtx=False):
        self.events = events
        self.nvtx = nvtx

    def begin(self, name):
        if self.nvtx:
            torch.cuda.nvtx.range_push(f"maskgs:{name}")
        if self.events is not None and name in self.events:
            self.events[name][0].record()

    def end(self, name):
        if self.events is not None and name in self.events:
            self.events[name][1].record()
        if self.nvtx:
            torch.cuda.nvtx.range_pop()


class Rasterizer:
    """Owns the device buffers of one masked forward+backward and issues the
    C-ABI calls on the current torch stream."""

    def __init__(self, device="cuda", capacity: int = 0, capacity_headroom: float = 1.25,
                 tile_order: bool = True, validate: bool = False, nvtx: bool | None = None):
        self.device = torch.device(device)
        self.tile_order = tile_order
        # check the sorted tile lists against their bounds (mg_validate_lists)
        # before any render call reads them
        self.validate = validate
        # NVTX ranges per stage (maskgs:preprocess, :bin, :sort, :render, :loss,
        # :render_bwd, :preprocess_bwd), or MASKGS_NVTX=1
        self.nvtx = nvtx if nvtx is not None else os.environ.get("MASKGS_NVTX", "") == "1"
        self.capacity = int(capacity)
        self.headroom = capacity_headroom
        self._buf = {}
        self.status = torch.zeros(2, dtype=torch.int64, device=self.device)   # mg_status_word
        self.frag_count = torch.zeros(4, dtype=torch.int64, device=self.device)
        self.bwd_count = torch.zeros(6, dtype=torch.int64, device=self.device)
        self.num_instances = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.num_sorted = torch.zeros(1, dtype=torch.int64, device=self.device)
        self._l1_fused = False
        self._sort_mode = "radix8"
        # records of the 2D-gradient accumulator that a fused training forward
        # reset (0: none); the first backward after it only accumulates
        self._grad2d_reset_R = 0

    # -- buffers -------------------------------------------------------------
    def _get(self, name, numel, dtype):
        t = self._buf.get(name)
        if t is None or t.numel() < numel or t.dtype != dtype:
            t = torch.empty(max(int(numel), 1), dtype=dtype, device=self.device)
            self._buf[name] = t
        return t[:max(int(numel), 1)]

    def _stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _splats(self, R, n, V):
        s = abi.mg_splats()
        s.mask_count = self._get("mask_count", V, torch.int32).data_ptr()
        s.record = self._get("record", R * abi.MG_RECORD_FLOATS, torch.float32).data_ptr()
        s.tiles_touched = self._get("tiles", R, torch.int32).data_ptr()
        s.radius = self._get("radius", R, torch.int32).data_ptr()
        s.clamp = self._get("clamp", R, torch.uint8).data_ptr()
        s.bin_record = self._get("bin_record", 12 * R, torch.float32).data_ptr()
        s.mask = self._get("mask", n, torch.uint8).data_ptr()
        s.mask_soft = self._get("mask_soft", n, torch.float32).data_ptr()
        s.depth_key = self._get("depth_key", R, torch.int32).data_ptr()
        return s

    def _ensure_sort_buffers(self, cap, key_bits, tiles, bucket):
        self._get("keys", cap, torch.int32)
        self._get("vals", cap, torch.int32)
        self._get("keys_alt", cap, torch.int32)
        self._get("vals_alt", cap, torch.int32)
        ws = (abi.mg_sort_by_tile_workspace_bytes(cap, tiles) if bucket
              else abi.mg_sort_workspace_bytes(cap, key_bits))
        self._get("sort_ws", ws, torch.uint8)

    # -- forward --------------------------------------------------------------
    def forward(self, params: dict, cams, cfg: RasterConfig, view_ranges=None, check=True,
                count_fragments=False, stage_events=None, inference=False, l1_target=None):
        """Masked forward.  Returns the concatenated images (flat float32,
        per view [3][H][W]).  ``inference``: the forward-only renderer of a
        (pruned) model -- every Gaussian present, no state for a backward.
        ``l1_target`` (flat float32 like the images): the render kernel also
        takes the L1 loss against it (see ``forward_l1``)."""
        if inference:
            cfg = RasterConfig(**{**cfg.__dict__, "mask_mode": abi.MG_MASK_ALL_ONES,
                                  "given_mask": None, "lambda_m": 0.0})
        n = int(params["means"].shape[0])
        sh_degree = int(round(math.sqrt(params["sh"].shape[1]))) - 1
        ranges = view_ranges if view_ranges is not None else [(0, n)] * len(cams)
        views = make_views(cams, ranges)
        V = len(cams)
        ccfg = cfg.c()
        g = _gaussians_struct(params, sh_degree)
        R = sum(int(r[1]) for r in ranges)
        pix = sum(int(c.width) * int(c.height) for c in cams)
        tiles = abi.mg_total_tiles(views, V, ccfg)
        key_bits = abi.mg_tile_bits(views, V, ccfg)
        stream = self._stream()
        ev = _Events(stage_events, self.nvtx)
        self.status.zero_()
        if l1_target is not None and not count_fragments:
            # the fused render adds to the loss: zeroed here, ahead of the
            # kernels, so that nothing but kernels runs between them
            self._get("loss", 1, torch.float32).zero_()
        splats = self._splats(R, n, V)
        ev.begin("preprocess")
        abi.mg_preprocess(g, views, V, ccfg, splats, self.status, stream)
        ev.end("preprocess")
        bucket = cfg.sort == "bucket"
        ev.begin("bin")
        if bucket:
            # instances in record order; each tile's list is put in depth
            # order by the sort itself
            order = None
            self._buf.pop("order", None)
        else:
            # depth order of the records, then instances in that order
            order = self._get("order", R, torch.int32)
            dws = self._get("depth_ws", abi.mg_depth_order_workspace_bytes(R), torch.uint8)
            abi.mg_depth_order(splats, views, V, ccfg, order,
                               self._get("order_alt", R, torch.int32),
                               self._get("dkeys", R, torch.int32),
                               self._get("dkeys_alt", R, torch.int32),
                               dws, dws.numel(), self.status, stream)
        offsets = self._get("offsets", R, torch.int32)
        bin_ws = self._get("bin_ws", abi.mg_bin_workspace_bytes(R), torch.uint8)
        if self.capacity <= 0:
            # size the instance buffers from this step's own count
            abi.mg_bin(splats, views, V, ccfg, order, offsets, None, None, 0, self.num_instances,
                       bin_ws, bin_ws.numel(), self.status, stream)
            k = int(self.num_instances.item())
            self.capacity = max(int(k * self.headroom), 1024)
            self.status.zero_()
        self._ensure_sort_buffers(self.capacity, key_bits, tiles, bucket)
        abi.mg_bin(splats, views, V, ccfg, order, offsets, self._buf["keys"], self._buf["vals"],
                   self.capacity, self.num_instances, bin_ws, bin_ws.numel(), self.status, stream)
        ev.end("bin")
        if check:
            st = abi.mg_read_status(self.status, stream)
            if st.status == abi.MG_ERR_CAPACITY:
                self.capacity = int(st.required * self.headroom) + 1024
                self._ensure_sort_buffers(self.capacity, key_bits, tiles, bucket)
                self.status.zero_()
                abi.mg_bin(splats, views, V, ccfg, order, offsets, self._buf["keys"],
                           self._buf["vals"], self.capacity, self.num_instances, bin_ws,
                           bin_ws.numel(), self.status, stream)
            elif st.status != abi.MG_OK:
                raise abi.MaskgsError("mg_bin", st.status)
        ranges_buf = self._get("ranges", 2 * tiles, torch.int32)
        sort_ws = self._buf["sort_ws"]
        ev.begin("sort")
        if bucket:
            # one counting pass over the whole tile id, then each tile's list
            # in depth order
            abi.mg_sort_by_tile(self._buf["keys"], self._buf["vals"], splats.depth_key,
                                self.num_instances, self.capacity, tiles, self._buf["vals_alt"],
                                ranges_buf, sort_ws, sort_ws.numel(), self.num_sorted,
                                self.status, stream)
            sorted_vals = self._buf["vals_alt"]
        else:
            # instances arrive in depth order: a stable sort by tile id suffices
            alt = abi.mg_sort(self._buf["keys"], self._buf["vals"], self._buf["keys_alt"],
                              self._buf["vals_alt"], self.num_instances, self.capacity, key_bits,
                              ranges_buf, tiles, sort_ws, sort_ws.numel(), self.num_sorted,
                              self.status, stream)
            sorted_vals = self._buf["vals_alt"] if alt else self._buf["vals"]
        ev.end("sort")
        if self.validate:
            abi.mg_validate_lists(sorted_vals, ranges_buf, tiles, self.num_sorted, self.capacity, R,
                                  self.status, stream)
            st = abi.mg_read_status(self.status, stream)
            if st.status != abi.MG_OK:
                raise abi.MaskgsError(f"tile lists (detail {st.detail}, at {st.required})",
                                      st.status)
        # longest tile lists first (launch order only)
        tile_order = self._get("tile_order", tiles, torch.int32) if self.tile_order else None
        if tile_order is not None:
            abi.mg_tile_order(ranges_buf, tiles, tile_order, stream)
        image = self._get("image", 3 * pix, torch.float32)
        # kernels of ours per forward: preprocess (with the depth keys); with
        # the radix sort: a workspace reset, histogram, offsets and 4 digit
        # passes of the depth order, a reset, scan, duplicate, a workspace
        # reset, histogram (clearing the ranges), offsets, one pass per tile
        # digit, ranges; with the bucket sort: a reset, scan, duplicate,
        # count, scan, scatter, order; then the tile order and the render
        sort_launches = 5 if bucket else 7 + 3 + 4 + (key_bits + 7) // 8
        self._fwd_launches = 1 + sort_launches + (2 if bucket else 0) + 1 + \
            (tile_order is not None)
        self._sort_mode = cfg.sort
        if inference:
            ev.begin("render")
            abi.mg_render_inference(splats, sorted_vals, ranges_buf, tile_order, views, V, ccfg,
                                    image, stream)
            ev.end("render")
            self._state = None
            if check:
                st = abi.mg_read_status(self.status, stream)
                if st.status != abi.MG_OK:
                    raise abi.MaskgsError("inference forward", st.status)
            return image
        final_T = self._get("final_T", pix, torch.float32)
        n_contrib = self._get("n_contrib", pix, torch.int32)
        if count_fragments:
            self.frag_count.zero_()
        fused = l1_target is not None and not count_fragments
        if fused:
            dimg = self._get("dL_dimage", 3 * pix, torch.float32)
            loss = self._buf["loss"][:1]           # zeroed before the preprocess
        ev.begin("render")
        if fused:
            # the render kernel also resets the backward's 2D-gradient accumulator
            grad2d = self._get("grad2d", max(R, 1) * abi.MG_GRAD2D_FLOATS, torch.float32)
            abi.mg_render_l1_reset2d(splats, sorted_vals, ranges_buf, tile_order, views, V, ccfg,
                                     image, final_T, n_contrib, l1_target, dimg, loss, grad2d,
                                     stream)
            self._grad2d_reset_R = R
        else:
            abi.mg_render(splats, sorted_vals, ranges_buf, tile_order, views, V, ccfg, image,
                          final_T, n_contrib, self.frag_count if count_fragments else None, stream)
        ev.end("render")
        self._l1_fused = fused
        self._state = dict(g=g, views=views, V=V, cfg=ccfg, splats=splats, R=R, n=n, pix=pix,
                           sorted_vals=sorted_vals, ranges=ranges_buf, tiles=tiles,
                           tile_order=tile_order,
                           sh_degree=sh_degree, params=params, cams=cams)
        if check:
            st = abi.mg_read_status(self.status, stream)
            if st.status != abi.MG_OK:
                raise abi.MaskgsError("masked forward", st.status)
        return image

    # -- loss -----------------------------------------------------------------
    def launches_per_step(self):
        return self._fwd_launches

    def backward_launches(self):
        # 2D-gradient reset (taken by the fused render when it ran), render, preprocess
        return 2 if self._l1_fused else 3

    def forward_l1(self, params: dict, cams, cfg: RasterConfig, target, view_ranges=None,
                   check=True, count_fragments=False, stage_events=None):
        """The masked forward with the L1 render loss taken by the render
        kernel itself: returns (image, L, dL/dimage), L = L_render (L1) +
        lambda_m L_m (Eq. 8; the mask loss only when lambda_m != 0, its
        gradient added by the backward)."""
        image = self.forward(params, cams, cfg, view_ranges=view_ranges, check=check,
                             count_fragments=count_fragments, stage_events=stage_events,
                             l1_target=target)
        if not self._l1_fused:                   # the counting variant: a separate pass
            loss, dimg = self.l1_loss_grad(image, target)
            return image, loss, dimg
        s = self._state
        ev = _Events(stage_events, self.nvtx)
        ev.begin("loss")
        loss = self._buf["loss"][:1]
        if s["cfg"].lambda_m != 0.0:
            abi.mg_mask_loss(s["splats"], s["views"], s["V"], s["cfg"], loss, self._stream())
        ev.end("loss")
        return image, loss, self._buf["dL_dimage"][:3 * s["pix"]]

    def l1_loss_grad(self, image, target):
        """L = L_render (L1) + lambda_m L_m (Eq. 8; the mask loss only when
        lambda_m != 0, its gradient is added by the backward) and dL/dimage."""
        s = self._state
        dimg = self._get("dL_dimage", 3 * s["pix"], torch.float32)
        loss = self._get("loss", 1, torch.float32)
        loss.zero_()
        abi.mg_l1_loss_grad(image, target, s["views"], s["V"], dimg, loss, self._stream())
        if s["cfg"].lambda_m != 0.0:
            abi.mg_mask_loss(s["splats"], s["views"], s["V"], s["cfg"], loss, self._stream())
        return loss, dimg

    def mask_loss(self):
        """lambda_m L_m of the last forward (Eq. 7-8), a device scalar."""
        s = self._state
        loss = self._get("mask_loss", 1, torch.float32)
        loss.zero_()
        abi.mg_mask_loss(s["splats"], s["views"], s["V"], s["cfg"], loss, self._stream())
        return loss

    # -- state handed to a pending backward -------------------------------------
    # Buffers a backward reads: the splat records and per-Gaussian mask state,
    # the sorted instance lists, tile ranges and launch order, and the
    # per-pixel final transmittance and stop index.
    _STATE_BUFFERS = ("record", "tiles", "radius", "clamp", "bin_record", "mask", "mask_soft",
                      "mask_count", "depth_key", "keys", "vals", "keys_alt", "vals_alt",
                      "ranges", "tile_order", "final_T", "n_contrib")

    def take_state(self) -> dict:
        """Detach the last forward's state from this Rasterizer: the buffers
        it points into move to the returned state (the next forward allocates
        new ones), so a later forward cannot overwrite what a pending backward
        of this one reads.  Pass it to ``backward(state=...)``."""
        s = self._state
        if s is None:
            raise RuntimeError("take_state: no forward state (inference forwards keep none)")
        s = dict(s)
        s["buffers"] = {k: self._buf.pop(k) for k in self._STATE_BUFFERS if k in self._buf}
        self._state = None
        return s

    # -- backward -------------------------------------------------------------
    def backward(self, dL_dimage, out: dict | None = None, stage_events=None,
                 count_iterations=False, state: dict | None = None, lambda_m=None):
        """Gradients of <dL_dimage, image> (+ lambda_m L_m when the
        configuration's lambda_m is set) w.r.t. every parameter, overwritten
        into ``out`` when given.  ``state``: a forward's state from
        ``take_state`` (default: this Rasterizer's last forward).
        ``lambda_m``: overrides the weight of the mask-loss gradient."""
        s = state if state is not None else self._state
        if s is None:
            raise RuntimeError("backward: no forward state (its state was taken, or the "
                               "forward was an inference forward)")
        buf = s["buffers"] if "buffers" in s else self._buf
        stream = self._stream()
        ev = _Events(stage_events, self.nvtx)
        cfg = s["cfg"]
        if lambda_m is not None and float(lambda_m) != cfg.lambda_m:
            cfg = abi.mg_raster_cfg.from_buffer_copy(cfg)
            cfg.lambda_m = float(lambda_m)
        grad2d = self._get("grad2d", s["R"] * abi.MG_GRAD2D_FLOATS, torch.float32)
        # the accumulator a fused training forward reset serves the first
        # backward after it (same stream, same buffer); any other backward
        # resets it itself
        reset = 0 < s["R"] <= self._grad2d_reset_R
        self._grad2d_reset_R = 0
        ev.begin("render_bwd")
        if count_iterations:
            self.bwd_count.zero_()
        render_bwd = abi.mg_render_backward_accumulate if reset else abi.mg_render_backward
        render_bwd(s["splats"], s["sorted_vals"], s["ranges"], s["tile_order"], s["views"],
                   s["V"], cfg, buf["final_T"], buf["n_contrib"], dL_dimage, grad2d,
                   self.bwd_count if count_iterations else None, stream)
        if out is None:
            out = {k: torch.empty(s["params"][k].shape, dtype=torch.float32, device=self.device)
                   for k in PARAM_NAMES}
        ev.end("render_bwd")
        pg = abi.mg_param_grads()
        for k in PARAM_NAMES:
            setattr(pg, k, out[k].data_ptr())
        ev.begin("preprocess_bwd")
        abi.mg_preprocess_backward(s["g"], s["views"], s["V"], cfg, s["splats"], grad2d, pg,
                                   stream)
        ev.end("preprocess_bwd")
        return out

    # -- views of the forward state -------------------------------------------
    def splat_outputs(self):
        s = self._state
        R, n = s["R"], s["n"]
        order = self._buf["order"][:R] if "order" in self._buf else None
        return dict(record=self._buf["record"][:R * 12].view(R, 12), order=order,
                    tiles=self._buf["tiles"][:R], radius=self._buf["radius"][:R],
                    clamp=self._buf["clamp"][:R], mask=self._buf["mask"][:n],
                    mask_soft=self._buf["mask_soft"][:n], offsets=self._buf["offsets"][:R],
                    mask_count=self._buf["mask_count"][:s["V"]],
                    sorted_vals=s["sorted_vals"], ranges=s["ranges"][:2 * s["tiles"]],
                    final_T=self._buf["final_T"][:s["pix"]],
                    n_contrib=self._buf["n_contrib"][:s["pix"]],
                    num_instances=self.num_instances, num_sorted=self.num_sorted,
                    grad2d=self._buf.get("grad2d"))

    def sorted_keys(self):
        """Tile id of every sorted instance (the bucket sort keeps the ids
        implicit in the ranges: rebuilt from them here)."""
        s = self._state
        if self._sort_mode == "bucket":
            r = s["ranges"][:2 * s["tiles"]].view(-1, 2).long()
            counts = r[:, 1] - r[:, 0]
            return torch.repeat_interleave(torch.arange(s["tiles"], device=self.device),
                                           counts).to(torch.int32)
        return self._buf["keys_alt"] if s["sorted_vals"] is self._buf["vals_alt"] else self._buf["keys"]


class MaskedRasterize(torch.autograd.Function):
    """(images, mask_loss) = MaskedRasterize.apply(means, log_scales, quats,
    opacity_logit, sh, mask_logits, rasterizer, cams, cfg, view_ranges).

    images: the concatenated per-view images (Eq. 3-4); mask_loss:
    lambda_m L_m of Eq. 7-8 (a 0-d tensor, zero when cfg.lambda_m is 0).  The
    backward is the hand-written one of libmaskgs: Eq. 6 and Appendix A for
    the mask, the chain rule to every parameter, and the straight-through
    Gumbel-softmax (Sec. 3.3) to the existence scores, the mask loss's
    gradient scaled by the gradient that reaches the mask-loss output.

    Each forward detaches its state from the Rasterizer (``take_state``), so
    several forwards may be pending on one Rasterizer before their backwards
    run, in any order."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, mask_logits, rast, cams, cfg,
                view_ranges):
        params = dict(means=means.detach(), log_scales=log_scales.detach(),
                      quats=quats.detach(), opacity_logit=opacity_logit.detach(),
                      sh=sh.detach(), mask_logits=mask_logits.detach())
        img = rast.forward(params, cams, cfg, view_ranges=view_ranges)
        ml = torch.zeros((), dtype=torch.float32, device=rast.device)
        if cfg.lambda_m != 0.0:
            ml = rast.mask_loss().reshape(()).clone()
        ctx.rast = rast
        ctx.state = rast.take_state()
        ctx.lambda_m = float(cfg.lambda_m)
        return img.clone(), ml

    @staticmethod
    def backward(ctx, dimg, dml):
        state = ctx.state
        lam = 0.0
        if ctx.lambda_m != 0.0 and dml is not None:
            lam = ctx.lambda_m * float(dml.item())
        if dimg is None:
            dimg = torch.zeros(3 * state["pix"], dtype=torch.float32, device=ctx.rast.device)
        out = ctx.rast.backward(dimg.contiguous().float(), state=state, lambda_m=lam)
        p = state["params"]
        # gradients are computed in FP32; autograd wants the parameters' dtype
        g = [out[k].to(p[k].dtype) for k in PARAM_NAMES]
        return (*g, None, None, None, None)


def rasterize(params: dict, cams, cfg: RasterConfig, rast: Rasterizer | None = None,
              view_ranges=None, return_mask_loss: bool = False):
    """Differentiable masked rasterisation of ``params`` (CUDA tensors: means
    and mask logits FP32, the other attributes FP32, BF16 or FP16) for
    ``cams``; returns a list of [3, H, W] images, and with
    ``return_mask_loss`` also lambda_m L_m (Eq. 7-8), a differentiable 0-d
    tensor to add to the render loss (Eq. 8)."""
    rast = rast or Rasterizer(params["means"].device)
    flat, ml = MaskedRasterize.apply(*(params[k] for k in PARAM_NAMES), rast, cams, cfg,
                                     view_ranges)
    out, o = [], 0
    for c in cams:
        n = 3 * c.width * c.height
        out.append(flat[o:o + n].view(3, c.height, c.width))
        o += n
    return (out, ml) if return_mask_loss else out
