"""Pins of the oracle's compositing (Eq. 1-4) and its backward (Eq. 6,
Appendix A) against brute force, the paper's invariants, closed forms and
central finite differences."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import binning, fp32_path, pipeline, render
from paper_2412_20522_gb300 import scenes


@pytest.fixture(scope="module")
def small():
    """A 48x40 frame (3x3 tiles with ragged edges) of 300 Gaussians."""
    g = scenes.uniform_gaussians(300, seed=7, log_scale_mu=-3.0)
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 48, 40, 40.0)
    cfg = pipeline.OracleConfig(bg=(0.2, 0.5, 0.9))
    views, M, minfo = pipeline.forward(g, [cam], cfg)
    return g, cam, cfg, views[0], M


def _rect(fp):
    return np.stack([fp["x0"], fp["x1"], fp["y0"], fp["y1"]], 1).astype(np.int32)


def test_tiled_equals_bruteforce_bitwise(small):
    """The tiled render over the filtered tile lists equals the per-pixel
    brute force over every Gaussian whose rectangle covers the pixel's tile,
    bit for bit: the tile filter drops only pairs under the alpha floor in the
    whole tile.  (The stop index counts list positions, which the filter
    removes, so it can only shrink.)"""
    g, cam, cfg, v, M = small
    for masked in (0, 1):
        t = render.render_tiled(v.splats, cam.width, cam.height, 16, 16, v.sorted_vals,
                                v.ranges, cfg.bg, masked)
        b = render.render_bruteforce(v.splats, cam.width, cam.height, 16, 16, _rect(v.fp32),
                                     v.fp32["depth_bits"], cfg.bg, masked)
        for k in ("image", "final_T", "flags"):
            assert np.array_equal(t[k], b[k]), k
        assert (t["n_contrib"] <= b["n_contrib"]).all()
        assert (t["n_contrib"] < b["n_contrib"]).any()


def test_all_ones_mask_is_plain_3dgs_bitwise(small):
    """Eq. 3-4 with M = 1 everywhere reduce to Eq. 1-2."""
    g, cam, cfg, v, M = small
    sp = v.splats
    ones = render.SplatsF64(sp.mean2d, sp.conic, sp.opacity, sp.rgb, np.ones(sp.n))
    a = render.render_tiled(ones, cam.width, cam.height, 16, 16, v.sorted_vals, v.ranges,
                            cfg.bg, masked=1)
    b = render.render_tiled(ones, cam.width, cam.height, 16, 16, v.sorted_vals, v.ranges,
                            cfg.bg, masked=0)
    assert np.array_equal(a["image"], b["image"]) and np.array_equal(a["final_T"], b["final_T"])


def test_masked_gaussian_equals_deleted_bitwise(small):
    """M_i = 0 acts as pruned (Sec. 3.3): same image as removing Gaussian i."""
    g, cam, cfg, v, M = small
    off = np.nonzero(M == 0)[0]
    assert off.size > 50
    rect = _rect(v.fp32)
    masked = render.render_bruteforce(v.splats, cam.width, cam.height, 16, 16, rect,
                                      v.fp32["depth_bits"], cfg.bg, 1)
    sp = v.splats
    ones = render.SplatsF64(sp.mean2d, sp.conic, sp.opacity, sp.rgb, np.ones(sp.n))
    rect_del = rect.copy()
    rect_del[off] = (0, -1, 0, -1)                 # empty rectangle: never listed
    deleted = render.render_bruteforce(ones, cam.width, cam.height, 16, 16, rect_del,
                                       v.fp32["depth_bits"], cfg.bg, 1)
    assert np.array_equal(masked["image"], deleted["image"])
    assert np.array_equal(masked["final_T"], deleted["final_T"])


def test_weights_and_final_transmittance_sum_to_one(small):
    g, cam, cfg, v, M = small
    sp = v.splats
    white = render.SplatsF64(sp.mean2d, sp.conic, sp.opacity, np.ones((sp.n, 3)), sp.mask)
    out = render.render_tiled(white, cam.width, cam.height, 16, 16, v.sorted_vals, v.ranges,
                              (0.0, 0.0, 0.0), 1)
    assert np.abs(out["image"][0] + out["final_T"] - 1.0).max() < 1e-12
    assert out["final_T"].min() >= 1e-4 * (1 - 0.99) and out["final_T"].max() <= 1.0


def _single(opacity, M, rgb, bg, offset=(0.0, 0.0), conic=(0.5, 0.0, 0.5)):
    sp = render.SplatsF64(np.array([[8.5 + offset[0], 8.5 + offset[1]]]), np.array([conic]),
                          np.array([opacity]), np.array([rgb]), np.array([M]))
    return render.render_tiled(sp, 16, 16, 16, 16, np.array([0], np.uint32),
                               np.array([[0, 1]], np.uint32), bg, 1)


def test_single_gaussian_closed_form():
    """One Gaussian centred on a pixel centre: C = M min(.99, o) c + (1 - M alpha) c_bg."""
    for o, M in [(0.7, 1.0), (0.7, 0.0), (1.5, 1.0), (0.002, 1.0)]:
        out = _single(o, M, (0.2, 0.4, 0.8), (1.0, 0.5, 0.25))
        a = min(0.99, o) if min(0.99, o) >= 1 / 255 else 0.0
        expect = np.array([M * a * c + (1 - M * a) * b
                           for c, b in zip((0.2, 0.4, 0.8), (1.0, 0.5, 0.25))])
        assert np.allclose(out["image"][:, 8, 8], expect, atol=1e-15)


def test_worked_three_gaussian_example():
    """Three Gaussians centred on one pixel (power = 0, so alpha_i = o_i) with
    exact rational opacities; the middle one masked.  Expected values follow
    Eq. 3-4 and Appendix A by hand:
      alpha = (1/2, 1/4, 1/8), M = (1, 0, 1), c = (1, 1/2, 1/4) (grey), bg = 1
      T = (1, 1/2, 1/2), T_4 = 1/2 * 7/8 = 7/16
      C = 1/2*1 + 0 + 1/8*1/2*1/4 + 7/16 = 1/2 + 1/64 + 7/16 = 61/64
    With g = dL/dC = (1, 0, 0): b_4 = 0, b_3 = 1/8*1/4 = 1/32,
      b_2 = b_3 (masked), b_1 = 1/2 + 1/2 * 1/32 = 33/64
      dL/dM_3 = 1/8*1/2*(1/4 - 0) - 1/8*(7/16)/(7/8) = 1/64 - 1/16 = -3/64
      dL/dM_2 = 1/4*1/2*(1/2 - 1/32) - 1/4*(7/16)/1 = 15/256 - 7/64 = -13/256
      dL/dM_1 = 1/2*1*(1 - 1/32) - 1/2*(7/16)/(1/2) = 31/64 - 7/16 = 3/64
    """
    op = [0.5, 0.25, 0.125]
    Ms = [1.0, 0.0, 1.0]
    cs = [1.0, 0.5, 0.25]
    sp = render.SplatsF64(np.full((3, 2), 8.5), np.tile([[0.5, 0.0, 0.5]], (3, 1)),
                          np.array(op), np.array([[c] * 3 for c in cs]), np.array(Ms))
    vals = np.array([0, 1, 2], np.uint32)
    ranges = np.array([[0, 3]], np.uint32)
    out = render.render_tiled(sp, 16, 16, 16, 16, vals, ranges, (1.0, 1.0, 1.0), 1)
    assert out["image"][0, 8, 8] == float(Fraction(61, 64))
    assert out["final_T"][8, 8] == float(Fraction(7, 16))
    g = np.zeros((3, 16, 16))
    g[0, 8, 8] = 1.0
    gr = render.render_backward(sp, 16, 16, 16, 16, vals, ranges, g, (1.0, 1.0, 1.0))
    exp = [Fraction(3, 64), Fraction(-13, 256), Fraction(-3, 64)]
    assert gr["dmask"] == pytest.approx([float(x) for x in exp], abs=1e-15)
    assert gr["dalpha"][1] == 0.0                   # masked splat: no alpha gradient
    # dL/dc_i = M_i alpha_i T_i g
    assert gr["drgb"][:, 0] == pytest.approx([0.5, 0.0, 1 / 16], abs=1e-15)


def _loss(sp, cam, v, w, bg):
    out = render.render_tiled(sp, cam.width, cam.height, 16, 16, v.sorted_vals, v.ranges, bg, 1)
    return float((out["image"] * w).sum()), out


def test_backward_matches_central_differences(small):
    """Linear loss L = <w, C>.  C is affine in each M_i (Eq. 3-4), so its FD is
    exact up to rounding; the other inputs use h = 1e-6 and skip perturbations
    that change a discrete decision."""
    g, cam, cfg, v, M = small
    rng = np.random.default_rng(3)
    w = rng.standard_normal((3, cam.height, cam.width))
    base = v.splats
    gr = render.render_backward(base, cam.width, cam.height, 16, 16, v.sorted_vals, v.ranges,
                                w, cfg.bg)
    _, out0 = _loss(base, cam, v, w, cfg.bg)
    fields = dict(mean2d=base.mean2d, conic=base.conic, opacity=base.opacity,
                  rgb=base.rgb, mask=base.mask)
    gname = dict(mean2d="dmean2d", conic="dconic", opacity="dopacity", rgb="drgb",
                 mask="dmask")
    checked = 0
    for name, arr in fields.items():
        flat = arr.reshape(-1)
        cand = [i for i in range(flat.size) if (i // (flat.size // base.n)) in set(v.visible)]
        for i in rng.choice(cand, 40, replace=False):
            h = 0.25 if name == "mask" else 1e-6 * max(1.0, abs(flat[i]))
            res = []
            for sgn in (1, -1):
                pert = {k: a.copy() for k, a in fields.items()}
                pert[name].reshape(-1)[i] += sgn * h
                sp = render.SplatsF64(**pert)
                L, out = _loss(sp, cam, v, w, cfg.bg)
                res.append((L, out))
            if any(not np.array_equal(o["n_contrib"], out0["n_contrib"]) for _, o in res):
                continue
            fd = (res[0][0] - res[1][0]) / (2 * h)
            an = gr[gname[name]].reshape(-1)[i]
            assert fd == pytest.approx(an, rel=1e-5, abs=1e-8), (name, i)
            checked += 1
    assert checked > 150


def test_masked_splats_get_no_alpha_gradient(small):
    g, cam, cfg, v, M = small
    rng = np.random.default_rng(4)
    w = rng.standard_normal((3, cam.height, cam.width))
    gr = render.render_backward(v.splats, cam.width, cam.height, 16, 16, v.sorted_vals,
                                v.ranges, w, cfg.bg)
    off = M == 0
    assert (gr["dalpha"][off] == 0).all() and (gr["dopacity"][off] == 0).all()
    assert (gr["dmean2d"][off] == 0).all() and (gr["drgb"][off] == 0).all()
    assert np.count_nonzero(gr["dmask"][off]) > 20       # but they do get dL/dM


def test_background_term_vanishes_for_black_bg(small):
    """With c_bg = 0 Appendix A's second term drops and Eq. 6 alone remains."""
    g, cam, cfg, v, M = small
    w = np.random.default_rng(5).standard_normal((3, cam.height, cam.width))
    a = render.render_backward(v.splats, cam.width, cam.height, 16, 16, v.sorted_vals,
                               v.ranges, w, (0.0, 0.0, 0.0))
    b = render.render_backward(v.splats, cam.width, cam.height, 16, 16, v.sorted_vals,
                               v.ranges, w, cfg.bg)
    assert not np.allclose(a["dmask"], b["dmask"])
    assert np.allclose(a["drgb"], b["drgb"])             # colour gradient has no bg term


def test_binning_sort_and_ranges(small):
    g, cam, cfg, v, M = small
    assert v.K == int(v.fp32["tiles"].astype(np.int64).sum())
    assert 0 < v.K_kept < v.K                             # the tile filter drops some pairs
    assert np.array_equal(np.sort(v.vals[v.keep]), np.sort(v.sorted_vals))   # a permutation
    k = v.sorted_keys
    assert (k[1:] >= k[:-1]).all()
    # ties in key keep Gaussian-index order
    same = k[1:] == k[:-1]
    assert (v.sorted_vals[1:][same] > v.sorted_vals[:-1][same]).all()
    r = v.ranges.astype(np.int64)
    assert (r[:, 1] - r[:, 0]).sum() == v.K_kept
    cover = np.zeros(v.K_kept, int)
    for t, (s, e) in enumerate(r):
        assert ((k[s:e] >> np.uint64(32)) == t).all()
        cover[s:e] += 1
    assert (cover == 1).all()
