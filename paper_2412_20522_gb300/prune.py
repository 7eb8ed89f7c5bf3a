"""Pruning of Sec. 3.5 on the GPU: n mask draws per Gaussian (the paper: 10),
keep the Gaussians sampled present at least once, compact every attribute
array to the survivors (order kept).  Both steps run in libmaskgs."""
from __future__ import annotations

import ctypes as C
import math

import torch

from . import abi
from .rasterize import PARAM_NAMES, _gaussians_struct


def _stream(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _struct(params):
    sh_degree = int(round(math.sqrt(params["sh"].shape[1]))) - 1
    return _gaussians_struct(params, sh_degree)


def prune_sample(params: dict, seed: int, iteration: int, n_draws: int = 10) -> torch.Tensor:
    """keep[i] (uint8 0/1): Gaussian i sampled present in at least one of
    n_draws draws (Philox draws 1..n_draws of the training noise stream)."""
    dev = params["means"].device
    keep = torch.empty(int(params["means"].shape[0]), dtype=torch.uint8, device=dev)
    abi.mg_prune_sample(_struct(params), int(seed), int(iteration), int(n_draws), keep,
                        _stream(dev))
    return keep


class Compactor:
    """Reusable buffers for mg_compact (destination arrays, index, workspace)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.n_kept = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.status = torch.zeros(2, dtype=torch.int64, device=self.device)
        self._ws = None
        self.dst = None
        self.new_index = None

    def run(self, params: dict, keep: torch.Tensor):
        """Enqueue the compaction (no synchronisation).  The survivors are the
        first n_kept rows of ``self.dst``."""
        n = int(params["means"].shape[0])
        if self.dst is None or self.dst["means"].shape[0] != n or any(
                self.dst[k].dtype != params[k].dtype or self.dst[k].shape != params[k].shape
                for k in PARAM_NAMES):
            self.dst = {k: torch.empty_like(params[k]) for k in PARAM_NAMES}
            self.new_index = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        wsb = abi.mg_compact_workspace_bytes(n)
        if self._ws is None or self._ws.numel() < wsb:
            self._ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=self.device)
        arr = abi.mg_gaussian_arrays()
        for k in PARAM_NAMES:
            setattr(arr, k, self.dst[k].data_ptr())
        self.status.zero_()
        abi.mg_compact(_struct(params), keep, arr, self.new_index, self.n_kept, self._ws,
                       self._ws.numel(), self.status, _stream(self.device))

    def result(self, clone: bool = True):
        """(survivor params, new_index) after synchronising on the count."""
        st = abi.mg_read_status(self.status, _stream(self.device))
        if st.status != abi.MG_OK:
            raise abi.MaskgsError("mg_compact", st.status)
        k = int(self.n_kept.item())
        out = {name: (t[:k].clone() if clone else t[:k]) for name, t in self.dst.items()}
        return out, self.new_index[:self.dst["means"].shape[0]]


def prune(params: dict, seed: int, iteration: int, n_draws: int = 10):
    """Sample, then compact: returns (survivor params, new_index int32 [n],
    keep uint8 [n])."""
    keep = prune_sample(params, seed, iteration, n_draws)
    c = Compactor(params["means"].device)
    c.run(params, keep)
    out, new_index = c.result()
    return out, new_index, keep
