"""mg_bin_noalloc, the binning entry point for callers that cannot allocate
device memory (its scratch is a fixed array inside the library), gives the
same instance offsets, count, keys and values as mg_bin with a caller
workspace -- on two calls in a row, since the array keeps the previous
call's contents.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def _splat(g, cams):
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    rast = Rasterizer()
    rast.forward(to_device(g), cams, RasterConfig())
    torch.cuda.synchronize()
    return rast


def _bin(abi, rast, noalloc, ordered=True):
    s = rast._state
    order = rast.splat_outputs()["order"] if ordered else None
    R = s["R"]
    dev = rast.device
    cap = rast.capacity
    offsets = torch.full((R,), -1, dtype=torch.int32, device=dev)
    keys = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    vals = torch.full((cap,), -1, dtype=torch.int32, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = rast._stream()
    if noalloc:
        abi.mg_bin_noalloc(s["splats"], s["views"], s["V"], s["cfg"], order, offsets, keys, vals,
                           cap, n, status, stream)
    else:
        ws = torch.empty(abi.mg_bin_workspace_bytes(R), dtype=torch.uint8, device=dev)
        abi.mg_bin(s["splats"], s["views"], s["V"], s["cfg"], order, offsets, keys, vals, cap, n,
                   ws, ws.numel(), status, stream)
    torch.cuda.synchronize()
    k = int(n.item())
    assert int(status[0].item()) == 0
    return offsets.cpu().numpy(), k, keys[:k].cpu().numpy(), vals[:k].cpu().numpy()


@pytest.mark.parametrize("which", ["tiny", "clusters"])
def test_noalloc_matches_workspace_binning_twice(which):
    from paper_2412_20522_gb300 import abi
    if which == "tiny":
        g, cams, _ = scenes.tiny_workload()
    else:
        g = scenes.cluster_gaussians(60_000, seed=4)
        cams = [scenes.ring_camera(0.0, 4.0, 300, 200, 230.0),
                scenes.ring_camera(1.0, 4.0, 200, 150, 180.0)]
    rast = _splat(g, cams)
    for ordered in (True, False):
        ref = _bin(abi, rast, noalloc=False, ordered=ordered)
        assert ref[1] > 0
        for _ in range(2):
            got = _bin(abi, rast, noalloc=True, ordered=ordered)
            assert got[1] == ref[1]
            assert np.array_equal(got[0], ref[0])
            assert np.array_equal(got[2], ref[2])
            assert np.array_equal(got[3], ref[3])


def test_noalloc_rejects_more_records_than_its_array_holds():
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, make_views
    g, cams, _ = scenes.tiny_workload(100)
    rast = _splat(g, cams)
    s = rast._state
    offsets = torch.zeros(16, dtype=torch.int32, device=rast.device)
    n = torch.zeros(1, dtype=torch.int64, device=rast.device)
    ok = make_views(cams, [(0, 1 << 24)])
    big = make_views(cams, [(0, (1 << 24) + 1)])
    # the size check comes first: nothing is launched for an oversized request
    with pytest.raises(abi.MaskgsError) as e:
        abi.mg_bin_noalloc(s["splats"], big, 1, RasterConfig().c(), None, offsets, None, None, 0,
                           n, None, rast._stream())
    assert e.value.status == abi.MG_ERR_INVALID_ARG
    assert abi.load().mg_bin_noalloc(None, ok, 1, RasterConfig().c(), None, None, None, None, 0,
                                     None, None, None) == abi.MG_ERR_INVALID_ARG


def test_noalloc_at_its_largest_size():
    """Exactly 2^24 records, the most the fixed array holds: the request passes
    the size check and its scan uses the array up to its last word.  Counting
    mode (capacity 0: offsets and the total only, no instance is written, and
    the status word reports MG_ERR_CAPACITY with the count needed), so only
    the tile counts are needed; the result equals mg_bin's, twice."""
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, make_views
    _, cams, _ = scenes.tiny_workload(100)
    dev = torch.device("cuda")
    R = 1 << 24
    gen = torch.Generator(device="cpu").manual_seed(7)
    tiles = torch.randint(0, 4, (R,), generator=gen, dtype=torch.int32).to(dev)
    dummy = torch.zeros(16, dtype=torch.float32, device=dev)     # not read in counting mode
    s = abi.mg_splats()
    s.tiles_touched = tiles.data_ptr()
    s.bin_record = dummy.data_ptr()
    views = make_views(cams, [(0, R)])
    cfg = RasterConfig().c()
    stream = C_stream()
    ws = torch.empty(abi.mg_bin_workspace_bytes(R), dtype=torch.uint8, device=dev)
    results = []
    for noalloc in (False, True, True):
        offsets = torch.full((R,), -1, dtype=torch.int32, device=dev)
        n = torch.zeros(1, dtype=torch.int64, device=dev)
        status = torch.zeros(2, dtype=torch.int64, device=dev)
        if noalloc:
            abi.mg_bin_noalloc(s, views, 1, cfg, None, offsets, None, None, 0, n, status, stream)
        else:
            abi.mg_bin(s, views, 1, cfg, None, offsets, None, None, 0, n, ws, ws.numel(), status,
                       stream)
        torch.cuda.synchronize()
        word = status.cpu().numpy()
        assert int(word[0]) & 0xFFFFFFFF == abi.MG_ERR_CAPACITY
        assert int(word[1]) == int(n.item())
        results.append((int(n.item()), offsets.cpu().numpy()))
    assert results[0][0] == int(tiles.sum().item())
    for k, off in results[1:]:
        assert k == results[0][0]
        assert np.array_equal(off, results[0][1])


def C_stream():
    import ctypes
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
