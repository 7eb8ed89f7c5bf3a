"""Bounds checks in place of a memory sanitiser.

* mg_validate_lists on the tile lists of both sort forms and both binning
  modes: clean; on copies corrupted on the host (within their buffers): an
  overlapping range, a range past the instance count, a record index past R,
  a wrong instance count -- each raises MG_ERR_BOUNDS with its detail.
* The debug build (MG_DEBUG_BOUNDS, in a subprocess with
  MASKGS_LIBRARY=debug): a clean step reports nothing and gives the oracle's
  lists; an order array holding a record index past R -- a caller error the
  ordinary build would follow out of the array -- is caught in the binning
  kernels (MG_ERR_BOUNDS, detail 1, the bad index) and its slots dropped.
  Only the debug build is ever given that input.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _forward(g, cams, **kw):
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    rast = Rasterizer(validate=True)
    rast.forward(to_device(g), cams, RasterConfig(**kw))
    torch.cuda.synchronize()
    return rast


def _validate(abi, rast, vals, ranges, num_sorted):
    s = rast._state
    status = torch.zeros(2, dtype=torch.int64, device="cuda")
    abi.mg_validate_lists(vals, ranges, s["tiles"], num_sorted, rast.capacity, s["R"], status,
                          rast._stream())
    return abi.mg_read_status(status, rast._stream())


@pytest.mark.parametrize("kw", [dict(), dict(sort="bucket"), dict(bin_mode=1),
                                dict(sort="bucket", tile_w=32, tile_h=8)])
def test_valid_lists_pass(kw):
    from paper_2412_20522_gb300 import abi
    g = scenes.cluster_gaussians(60_000, seed=14)
    cams = [scenes.ring_camera(0.7, 4.0, 320, 200, 240.0),
            scenes.ring_camera(2.2, 4.0, 200, 160, 180.0)]
    rast = _forward(g, cams, **kw)                 # validate=True checks inside forward
    so = rast.splat_outputs()
    st = _validate(abi, rast, so["sorted_vals"], so["ranges"], rast.num_sorted)
    assert st.status == abi.MG_OK


def test_corrupted_lists_are_reported():
    from paper_2412_20522_gb300 import abi
    g, cams, _ = scenes.tiny_workload()
    rast = _forward(g, cams)
    so = rast.splat_outputs()
    vals0 = so["sorted_vals"].clone()
    ranges0 = so["ranges"].clone()
    n = int(rast.num_sorted.item())
    R = rast._state["R"]
    r = ranges0.cpu().numpy().reshape(-1, 2)
    ne = np.nonzero(r[:, 1] > r[:, 0])[0]
    assert ne.size >= 3 and n > 10

    # a range reaching back into the previous non-empty one
    bad = r.copy()
    bad[ne[2], 0] = bad[ne[1], 0]
    st = _validate(abi, rast, vals0, torch.as_tensor(bad.reshape(-1)).cuda(), rast.num_sorted)
    assert (st.status, st.detail) == (abi.MG_ERR_BOUNDS, 7)
    # a range past the instance count
    bad = r.copy()
    bad[ne[-1], 1] = n + 1
    st = _validate(abi, rast, vals0, torch.as_tensor(bad.reshape(-1)).cuda(), rast.num_sorted)
    assert (st.status, st.detail) == (abi.MG_ERR_BOUNDS, 7)
    # a record index past R
    v = vals0.clone()
    v[n // 2] = R + 3
    st = _validate(abi, rast, v, ranges0, rast.num_sorted)
    assert (st.status, st.detail, st.required) == (abi.MG_ERR_BOUNDS, 8, n // 2)
    # an instance count the ranges do not add up to (still within capacity)
    wrong = rast.num_sorted.clone() - 1
    st = _validate(abi, rast, vals0, ranges0, wrong)
    assert st.status == abi.MG_ERR_BOUNDS and st.detail in (7, 9)


_DEBUG_SCRIPT = r"""
import json, sys
sys.path.insert(0, %(root)r); sys.path.insert(0, %(tests)r)
import numpy as np, torch
from paper_2412_20522_gb300 import abi, scenes
from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
from gpu_helpers import to_device
from oracle import pipeline
assert abi.lib_path().endswith("libmaskgs_debug.so")
g, cams, tgt = scenes.tiny_workload()
rast = Rasterizer(validate=True)
img = rast.forward(to_device(g), cams, RasterConfig())
loss, dimg = rast.l1_loss_grad(img, torch.as_tensor(tgt).cuda().reshape(-1))
rast.backward(dimg)
torch.cuda.synchronize()
clean = abi.mg_read_status(rast.status, rast._stream())
views, M, _ = pipeline.forward(g, cams, pipeline.OracleConfig())
so = rast.splat_outputs()
Ks = int(so["num_sorted"].item())
lists_equal = bool(np.array_equal(so["sorted_vals"][:Ks].cpu().numpy().view(np.uint32),
                                  views[0].sorted_vals.astype(np.uint32)))
# a caller's order array with one record index past R
s = rast._state
R = s["R"]
order = torch.arange(R, dtype=torch.int32, device="cuda")
order[5] = R + 7
offsets = torch.empty(R, dtype=torch.int32, device="cuda")
keys = torch.empty(rast.capacity, dtype=torch.int32, device="cuda")
vals = torch.empty(rast.capacity, dtype=torch.int32, device="cuda")
n = torch.zeros(1, dtype=torch.int64, device="cuda")
status = torch.zeros(2, dtype=torch.int64, device="cuda")
ws = torch.empty(abi.mg_bin_workspace_bytes(R), dtype=torch.uint8, device="cuda")
abi.mg_bin(s["splats"], s["views"], s["V"], s["cfg"], order, offsets, keys, vals, rast.capacity,
           n, ws, ws.numel(), status, rast._stream())
bad = abi.mg_read_status(status, rast._stream())
print(json.dumps({"clean": clean.status, "lists_equal": lists_equal, "bad_status": bad.status,
                  "bad_detail": bad.detail, "bad_index": int(bad.required), "R": R}))
"""


def test_debug_build_checks_bounds():
    from paper_2412_20522_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, MASKGS_LIBRARY="debug")
    code = _DEBUG_SCRIPT % {"root": ROOT, "tests": os.path.join(ROOT, "tests")}
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["clean"] == 0 and out["lists_equal"]
    assert out["bad_status"] == 6 and out["bad_detail"] == 1
    assert out["bad_index"] == out["R"] + 7


def test_nvtx_ranges_change_nothing():
    """Stage ranges for a profiler's timeline (Rasterizer(nvtx=True)): the same
    image and gradients as without them."""
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, tgt = scenes.tiny_workload(3000)
    p = to_device(g)
    t = torch.as_tensor(tgt).cuda().reshape(-1)
    out = []
    for nv in (False, True):
        rast = Rasterizer(nvtx=nv)
        img = rast.forward(p, cams, RasterConfig())
        _, dimg = rast.l1_loss_grad(img, t)
        gr = rast.backward(dimg)
        torch.cuda.synchronize()
        out.append((img.clone(), gr["sh"].clone()))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.allclose(out[0][1], out[1][1], rtol=1e-5, atol=1e-12)
