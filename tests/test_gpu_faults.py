"""Failure detection without a GPU fault: capacity overflow is reported with
the count needed (and the rasteriser's retry then gives the normal result);
a bounded device-side wait on a flag that nothing sets gives up and reports
a timeout, leaving the context usable; Gaussians with non-finite inputs are
culled as the oracle culls them."""
import numpy as np
import pytest
import torch

from gpu_helpers import to_device
from oracle import fp32_path
from paper_2412_20522_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_capacity_overflow_reported_then_retried():
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, _ = scenes.tiny_workload(6000)
    p = to_device(g)
    ref = Rasterizer()
    img_ref = ref.forward(p, cams, RasterConfig()).clone()
    K = int(ref.num_instances.item())
    # without the check the step is enqueued as is: the status word says why
    small = Rasterizer(capacity=K // 3)
    small.forward(p, cams, RasterConfig(), check=False)
    st = abi.mg_read_status(small.status, small._stream())
    assert st.status == abi.MG_ERR_CAPACITY and st.required == K
    assert int(small.num_sorted.item()) == 0            # nothing sorted
    # with the check the rasteriser grows its buffers and redoes the binning
    retry = Rasterizer(capacity=K // 3)
    img = retry.forward(p, cams, RasterConfig(), check=True)
    torch.cuda.synchronize()
    assert retry.capacity >= K
    assert torch.equal(img, img_ref)


def test_bounded_wait_times_out_and_context_stays_usable():
    from paper_2412_20522_gb300 import abi
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    status = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = Rasterizer()._stream()
    abi.mg_selftest_wait_timeout(1000, status, stream)
    st = abi.mg_read_status(status, stream)
    assert st.status == abi.MG_ERR_TIMEOUT and st.detail == 4
    assert abi.status_string(st.status) == "device-side wait timed out"
    # the warp-wide look-back of the single-pass scans
    status.zero_()
    abi.mg_selftest_warp_wait_timeout(1000, status, stream)
    st = abi.mg_read_status(status, stream)
    assert st.status == abi.MG_ERR_TIMEOUT and st.detail == 5
    # the same context renders normally afterwards
    g, cams, _ = scenes.tiny_workload(2000)
    r = Rasterizer()
    r.forward(to_device(g), cams, RasterConfig(), check=True)
    torch.cuda.synchronize()


def test_non_finite_gaussians_are_culled_like_the_oracle():
    from paper_2412_20522_gb300.rasterize import RasterConfig, Rasterizer
    g, cams, _ = scenes.tiny_workload(3000)
    g.means[5] = np.nan
    g.means[9, 2] = np.inf
    g.log_scales[17] = np.nan
    g.quats[23] = 0.0                       # no rotation
    g.quats[31] = np.nan
    rast = Rasterizer()
    img = rast.forward(to_device(g), cams, RasterConfig())
    torch.cuda.synchronize()
    with np.errstate(invalid="ignore"):
        fp = fp32_path.project32(g.means, g.log_scales, g.quats, cams[0], 16, 16)
        fp.update(fp32_path.candidate_rect(fp, 16, 16))
    so = rast.splat_outputs()
    assert np.array_equal(so["tiles"].cpu().numpy().view(np.uint32), fp["tiles"])
    assert np.array_equal(so["radius"].cpu().numpy(), fp["radius"])
    for i in (5, 9, 17, 23, 31):
        assert fp["tiles"][i] == 0
    assert np.isfinite(img.cpu().numpy()).all()
