"""Pins of the oracle's splat (Sec. 3.1) against closed forms, quadrature and
brute force: SH orthonormality, EWA special cases, the FP32 decision path
against its FP64 counterpart, and the tile-rectangle definition."""
import math

import numpy as np
import pytest
import torch

from oracle import fp32_path, preprocess
from paper_2412_20522_gb300 import scenes

DT = torch.float64


def _sphere_quadrature(nz=24, nphi=48):
    z, w = np.polynomial.legendre.leggauss(nz)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    W = np.repeat(w[:, None], nphi, 1) * (2 * np.pi / nphi)
    s = np.sqrt(1 - Z ** 2)
    d = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    return torch.as_tensor(d), torch.as_tensor(W.reshape(-1))


def test_sh_basis_orthonormal():
    d, w = _sphere_quadrature()
    Y = preprocess.sh_basis(d, 3)
    gram = (Y * w[:, None]).T @ Y
    assert torch.allclose(gram, torch.eye(16, dtype=DT), atol=1e-12)


def test_sh_basis_closed_forms():
    """Textbook values with the Condon-Shortley phase."""
    rng = np.random.default_rng(1)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = preprocess.sh_basis(torch.as_tensor(d), 2).numpy()
    x, y, z = d.T
    assert np.allclose(Y[:, 0], 0.5 / math.sqrt(math.pi))
    k1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 1], -k1 * y)
    assert np.allclose(Y[:, 2], k1 * z)
    assert np.allclose(Y[:, 3], -k1 * x)
    assert np.allclose(Y[:, 6], math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1))
    assert np.allclose(Y[:, 8], math.sqrt(15 / (16 * math.pi)) * (x * x - y * y))


def _one_gaussian(mean, log_s, quat, sh=None, opacity_logit=0.0):
    sh = np.zeros((1, 16, 3), np.float32) if sh is None else sh
    return scenes.Gaussians(np.array([mean], np.float32), np.array([log_s], np.float32),
                            np.array([quat], np.float32), np.array([opacity_logit], np.float32),
                            sh, np.zeros((1, 2), np.float32))


def _p64(g):
    return {k: torch.as_tensor(np.asarray(getattr(g, k), np.float64))
            for k in ("means", "log_scales", "quats", "opacity_logit", "sh")}


def _cam(W=128, H=96, f=100.0):
    return scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), W, H, f)


def test_isotropic_on_axis_closed_form():
    """An isotropic Gaussian of std s on the optical axis at depth z projects to
    Sigma_bar = ((f s / z)^2 + 0.3) I centred at the principal point."""
    cam = _cam()
    s = 0.05
    g = _one_gaussian((0.0, 0.0, 0.0), [math.log(s)] * 3, (0.3, -0.5, 0.7, 0.1))
    sp = preprocess.splat(_p64(g), cam)
    a, b, c = (t.item() for t in sp["cov"])
    s = math.exp(float(g.log_scales[0, 0]))          # the stored (float32) scale
    v = (cam.fx * s / 3.0) ** 2 + 0.3
    assert a == pytest.approx(v, rel=1e-12) and c == pytest.approx(v, rel=1e-12)
    assert abs(b) < 1e-12
    assert sp["mean2d"][0].tolist() == pytest.approx([cam.cx, cam.cy], abs=1e-12)
    assert sp["conic"][0].tolist() == pytest.approx([1 / v, 0.0, 1 / v], abs=1e-12)
    # the FP32 path agrees to FP32 precision
    d = fp32_path.project32(g.means, g.log_scales, g.quats, cam)
    assert float(d["a"][0]) == pytest.approx(v, rel=1e-6)
    assert abs(float(d["b"][0])) < 1e-6 * v
    assert int(d["radius"][0]) == math.ceil(3 * math.sqrt(v))


def test_identity_quaternion_axis_aligned():
    """q = (1,0,0,0) gives Sigma = S^2; for an identity camera rotation and a
    centred Gaussian, Sigma_bar = diag((f sx/z)^2, (f sy/z)^2) + 0.3 I."""
    cam = _cam()
    sx, sy, sz = 0.02, 0.07, 0.5
    g = _one_gaussian((0.0, 0.0, 0.0), [math.log(sx), math.log(sy), math.log(sz)],
                      (1.0, 0.0, 0.0, 0.0))
    sp = preprocess.splat(_p64(g), cam)
    a, b, c = (t.item() for t in sp["cov"])
    sx, sy = np.exp(g.log_scales[0, :2].astype(np.float64))
    assert a == pytest.approx((cam.fx * sx / 3) ** 2 + 0.3, rel=1e-12)
    assert c == pytest.approx((cam.fy * sy / 3) ** 2 + 0.3, rel=1e-12)
    assert abs(b) < 1e-12


def test_jacobian_of_offaxis_point_matches_finite_difference():
    """Sigma_bar - 0.3 I = J Sigma J^T with J the derivative of the pixel map
    at the Gaussian's centre (inside the 1.3 tan(fov/2) clamp)."""
    cam = _cam()
    mean = np.array([0.4, -0.25, 0.3])
    ls = np.log([0.03, 0.05, 0.04])
    q = np.array([0.9, 0.2, -0.3, 0.1])
    g = _one_gaussian(mean, ls, q)
    sp = preprocess.splat(_p64(g), cam)
    V = cam.viewmat.astype(np.float64)

    def pix(p):
        t = V[:, :3] @ p + V[:, 3]
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
    h = 1e-6
    J = np.stack([(pix(mean + h * e) - pix(mean - h * e)) / (2 * h) for e in np.eye(3)], 1)
    R = preprocess.quat_to_rot(torch.as_tensor(q[None])).numpy()[0]
    S = np.diag(np.exp(ls))
    cov = J @ R @ S @ S @ R.T @ J.T
    a, b, c = (t.item() for t in sp["cov"])
    assert np.allclose([a - 0.3, b, c - 0.3], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7)


def test_sh_degree0_colour():
    g = _one_gaussian((0.1, 0.2, 0.0), [-3.0] * 3, (1, 0, 0, 0),
                      sh=np.array([[[0.4, -0.2, 1.0]]], np.float32))
    sp = preprocess.splat(_p64(g), _cam())
    c0 = 0.5 / math.sqrt(math.pi)
    expect = np.maximum(np.array([0.4, -0.2, 1.0], np.float32).astype(np.float64) * c0 + 0.5, 0)
    assert np.allclose(sp["rgb"][0].numpy(), expect, atol=1e-15)
    g.sh[0, 0, 1] = -5.0
    sp = preprocess.splat(_p64(g), _cam())
    assert sp["rgb"][0, 1].item() == 0.0 and bool(sp["rgb_clamped"][0, 1])


def test_fp32_path_tracks_fp64():
    g, cams, _ = scenes.tiny_workload(2000)
    cam = cams[0]
    d = fp32_path.project32(g.means, g.log_scales, g.quats, cam)
    with torch.no_grad():
        sp = preprocess.splat(_p64(g), cam)
    vis = d["visible"]
    assert vis.sum() > 1000
    assert np.allclose(d["px"][vis], sp["mean2d"][vis, 0].numpy(), atol=1e-3)
    assert np.allclose(d["py"][vis], sp["mean2d"][vis, 1].numpy(), atol=1e-3)
    A, B, C = (t.numpy()[vis] for t in sp["cov"])
    scale = np.maximum(A, C)
    assert (np.abs(d["a"][vis] - A) / scale).max() < 1e-5
    assert (np.abs(d["b"][vis] - B) / scale).max() < 1e-5
    assert (np.abs(d["det"][vis] - sp["det"].numpy()[vis]) / sp["det"].numpy()[vis]).max() < 1e-4
    # radius from the FP64 eigenvalue agrees except within a rounding of the ceil
    mid = 0.5 * (A + C)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - sp["det"].numpy()[vis]))
    r64 = 3 * np.sqrt(lam)
    diff = d["radius"][vis] - np.ceil(r64)
    near = np.abs(r64 - np.round(r64)) < 1e-3
    assert (diff[~near] == 0).all()
    assert np.array_equal(d["depth_bits"].view(np.float32), d["tz"])


def test_near_plane_and_quaternion_culls():
    cam = _cam()
    g = scenes.Gaussians(
        np.array([[0, 0, -2.85], [0, 0, -2.75], [0, 0, 0]], np.float32),
        np.full((3, 3), -3.0, np.float32),
        np.array([[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 0]], np.float32),
        np.zeros(3, np.float32), np.zeros((3, 16, 3), np.float32), np.zeros((3, 2), np.float32))
    d = fp32_path.project32(g.means, g.log_scales, g.quats, cam)
    # z_cam = 0.15 (< 0.2 near plane), 0.25, and a zero quaternion
    assert d["visible"].tolist() == [False, True, False]
    assert d["tiles"].tolist()[0] == 0 and d["tiles"].tolist()[2] == 0
    assert d["radius"].tolist()[0] == 0


@pytest.mark.parametrize("tile", [(16, 16), (8, 32)])
def test_rect_is_tiles_overlapping_square(tile):
    """Brute force: tile (tx, ty) is in the rectangle iff its pixel span
    [tx*tw, (tx+1)*tw) x [ty*th, (ty+1)*th) meets the closed square
    [p - r, p + r]^2 and lies on the grid."""
    tw, th = tile
    g, cams, _ = scenes.tiny_workload(400)
    cam = cams[0]
    d = fp32_path.project32(g.means, g.log_scales, g.quats, cam, tw, th)
    gx, gy = d["grid"]
    px, py, r = d["px"].astype(np.float64), d["py"].astype(np.float64), d["radius"]
    for i in range(g.n):
        if r[i] == 0:
            assert d["tiles"][i] == 0
            continue
        # floor((p - r)/tw) <= tx <= floor((p + r)/tw) within the grid
        xs = [t for t in range(gx) if t * tw <= px[i] + r[i] and (t + 1) * tw > px[i] - r[i]]
        ys = [t for t in range(gy) if t * th <= py[i] + r[i] and (t + 1) * th > py[i] - r[i]]
        assert d["tiles"][i] == len(xs) * len(ys)
        if xs and ys:
            assert (d["x0"][i], d["x1"][i], d["y0"][i], d["y1"][i]) == (xs[0], xs[-1], ys[0], ys[-1])
