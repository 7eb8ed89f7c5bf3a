"""mg_bin with the depth order and the offsets at addresses that are not
16-byte aligned (views one element into larger buffers): the scan then reads
and writes them element by element instead of 128 bits at a time, and every
output -- offsets, instance count, keys and values -- equals the aligned
call's bit for bit."""
import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def _bin(abi, rast, shift):
    s = rast._state
    R, cap, dev = s["R"], rast.capacity, rast.device
    # the order and offset arrays `shift` elements into larger buffers
    order_buf = torch.zeros(R + 4, dtype=torch.int32, device=dev)
    order_buf[shift:shift + R] = rast.splat_outputs()["order"].view(torch.int32)
    order = order_buf[shift:shift + R]
    off_buf = torch.full((R + 4,), -1, dtype=torch.int32, device=dev)
    offsets = off_buf[shift:shift + R]
    keys = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    vals = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(2, dtype=torch.int64, device=dev)
    ws = torch.empty(abi.mg_bin_workspace_bytes(R), dtype=torch.uint8, device=dev)
    abi.mg_bin(s["splats"], s["views"], s["V"], s["cfg"], order, offsets, keys, vals, cap, n,
               ws, ws.numel(), status, rast._stream())
    torch.cuda.synchronize()
    k = int(n.item())
    assert int(status[0].item()) == 0
    # nothing written outside the view
    assert int(off_buf[:shift].ne(-1).sum()) == 0 and int(off_buf[shift + R:].ne(-1).sum()) == 0
    return offsets.cpu().numpy(), k, keys[:k].cpu().numpy(), vals[:k].cpu().numpy()


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_unaligned_order_and_offsets_bin_like_aligned(shift):
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g = scenes.cluster_gaussians(50_003, seed=9)      # a ragged last scan partition
    cams = [scenes.ring_camera(0.5, 4.0, 301, 203, 230.0)]
    rast = Rasterizer()
    rast.forward(to_device(g), cams, RasterConfig())
    torch.cuda.synchronize()
    ref = _bin(abi, rast, 0)
    got = _bin(abi, rast, shift)
    assert ref[1] > 0 and got[1] == ref[1]
    for a, b in zip(got[0:1] + got[2:], ref[0:1] + ref[2:]):
        assert np.array_equal(a, b)
