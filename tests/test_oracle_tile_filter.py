"""Pins of the decision path's tile filter (Sec. 3.1: only Gaussians whose
alpha reaches the floor take part in a tile's pixels).  A pair is dropped
only if the Gaussian's quadratic form exceeds 2 ln 255 at every pixel centre
of the tile -- checked here by evaluating it, in FP64, at all 256 centres --
and kept whenever some centre is clearly inside that ellipse."""
import math

import numpy as np

from oracle import fp32_path as fp

THR = 2 * math.log(255.0)


def _random_pairs(n, seed):
    rng = np.random.default_rng(seed)
    f32 = np.float32
    # covariances from random factors: round, elongated and needle-like
    s1 = np.exp(rng.uniform(-1, 5, n))
    s2 = s1 * np.exp(-rng.uniform(0, 9, n))                  # axis ratios up to e^9
    th = rng.uniform(0, np.pi, n)
    ct, st = np.cos(th), np.sin(th)
    a = ct * ct * s1 * s1 + st * st * s2 * s2 + 0.3
    b = ct * st * (s1 * s1 - s2 * s2)
    c = st * st * s1 * s1 + ct * ct * s2 * s2 + 0.3
    det = a * c - b * b
    px = rng.uniform(-40, 200, n)
    py = rng.uniform(-40, 200, n)
    tx = rng.integers(0, 10, n)
    ty = rng.integers(0, 10, n)
    d = dict(a=a.astype(f32), b=b.astype(f32), c=c.astype(f32), det=det.astype(f32),
             tiles=np.ones(n, np.uint32))
    return d, px.astype(f32), py.astype(f32), tx, ty


def _qmin_centres(a, b, c, det, px, py, tx, ty, tw=16, th=16):
    xs = tx[:, None] * tw + 0.5 + np.arange(tw)[None, :]
    ys = ty[:, None] * th + 0.5 + np.arange(th)[None, :]
    dx = xs[:, None, :] - px[:, None, None].astype(np.float64)
    dy = ys[:, :, None] - py[:, None, None].astype(np.float64)
    a, b, c, det = (np.asarray(v, np.float64)[:, None, None] for v in (a, b, c, det))
    q = (c * dx * dx - 2 * b * dx * dy + a * dy * dy) / det
    return q.reshape(q.shape[0], -1).min(1)


def test_dropped_pairs_are_under_the_floor_everywhere():
    d, px, py, tx, ty = _random_pairs(60_000, 1)
    tdet, rba, rbc = fp.tile_filter_params(d)
    keep = fp.tile_hit(px, py, d["a"], d["b"], d["c"], tdet, rba, rbc, tx, ty, 16, 16)
    qmin = _qmin_centres(d["a"], d["b"], d["c"], d["det"], px, py, tx, ty)
    assert (qmin[~keep] > THR).all(), qmin[~keep].min()
    # and a clear hit is never dropped
    assert keep[qmin < 0.99 * THR].all()
    # the filter does drop pairs the rectangle would keep
    assert 0.2 < (~keep).mean() < 0.95


def test_tile_shapes_and_needles():
    d, px, py, tx, ty = _random_pairs(20_000, 2)
    for tw, th in ((8, 32), (32, 8)):
        tdet, rba, rbc = fp.tile_filter_params(d)
        keep = fp.tile_hit(px, py, d["a"], d["b"], d["c"], tdet, rba, rbc, tx, ty, tw, th)
        qmin = _qmin_centres(d["a"], d["b"], d["c"], d["det"], px, py, tx, ty, tw, th)
        assert (qmin[~keep] > THR).all()
        assert keep[qmin < 0.99 * THR].all()


def test_centre_inside_tile_is_kept():
    n = 100
    d = dict(a=np.full(n, 0.31, np.float32), b=np.zeros(n, np.float32),
             c=np.full(n, 0.31, np.float32), det=np.full(n, 0.0961, np.float32),
             tiles=np.ones(n, np.uint32))
    tdet, rba, rbc = fp.tile_filter_params(d)
    px = np.full(n, 20.0, np.float32)
    py = np.full(n, 20.0, np.float32)
    tx = np.full(n, 1)
    ty = np.full(n, 1)
    assert fp.tile_hit(px, py, d["a"], d["b"], d["c"], tdet, rba, rbc, tx, ty, 16, 16).all()
    # a tiny Gaussian two tiles away is dropped
    tx2 = np.full(n, 3)
    assert not fp.tile_hit(px, py, d["a"], d["b"], d["c"], tdet, rba, rbc, tx2, ty, 16, 16).any()
