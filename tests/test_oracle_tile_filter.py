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


def _random_splats(n, seed, tw=16, th=16, gx=12, gy=10):
    """Random 2D splats (round to needle-like) with their 3-sigma tile
    rectangles on a gx x gy grid, as the decision path returns them."""
    d, px, py, _, _ = _random_pairs(n, seed)
    f32 = np.float32
    a, b, c = d["a"], d["b"], d["c"]
    mid = f32(0.5) * (a + c)
    hd = f32(0.5) * (a - c)
    lam = mid + np.sqrt(np.maximum(f32(0.1), hd * hd + b * b))
    rf = np.ceil(f32(3.0) * np.sqrt(lam))
    x0 = np.maximum(np.floor((px - rf) / f32(tw)), f32(0.0))
    x1 = np.minimum(np.floor((px + rf) / f32(tw)), f32(gx - 1))
    y0 = np.maximum(np.floor((py - rf) / f32(th)), f32(0.0))
    y1 = np.minimum(np.floor((py + rf) / f32(th)), f32(gy - 1))
    ok = (x0 <= x1) & (y0 <= y1)
    d.update(px=px, py=py, x0=np.where(ok, x0, 0).astype(np.int64),
             x1=np.where(ok, x1, -1).astype(np.int64), y0=np.where(ok, y0, 0).astype(np.int64),
             y1=np.where(ok, y1, -1).astype(np.int64))
    d["tiles"] = ((d["x1"] - d["x0"] + 1) * (d["y1"] - d["y0"] + 1)).astype(np.uint32)
    return d


def test_candidate_rectangle_holds_every_kept_tile():
    """Brute force over every tile of each 3-sigma rectangle: the filter keeps
    no tile outside the candidate rectangle, which lies inside the square."""
    for tw, th in ((16, 16), (8, 32), (32, 8)):
        d = _random_splats(3000, seed=11 + tw, tw=tw, th=th, gx=240 // tw + 1, gy=240 // th + 1)
        cand = fp.candidate_rect(d, tw, th)
        tdet, rba, rbc = fp.tile_filter_params(d)
        n_rect = n_cand = n_kept = 0
        for i in range(len(d["a"])):
            if d["tiles"][i] == 0:
                continue
            tys, txs = np.meshgrid(np.arange(d["y0"][i], d["y1"][i] + 1),
                                   np.arange(d["x0"][i], d["x1"][i] + 1), indexing="ij")
            tx, ty = txs.ravel(), tys.ravel()
            k = np.full(tx.shape, i)
            hit = fp.tile_hit(d["px"][k], d["py"][k], d["a"][k], d["b"][k], d["c"][k], tdet[k],
                              rba[k], rbc[k], tx, ty, tw, th)
            inside = ((tx >= cand["x0"][i]) & (tx <= cand["x1"][i]) &
                      (ty >= cand["y0"][i]) & (ty <= cand["y1"][i]))
            assert not (hit & ~inside).any(), (i, tw, th)
            assert cand["x0"][i] >= d["x0"][i] or cand["tiles"][i] == 0
            n_rect += tx.size
            n_cand += int(cand["tiles"][i])
            n_kept += int(hit.sum())
        assert n_kept <= n_cand < n_rect


def test_candidate_rectangle_of_round_splats_is_the_kept_box():
    """A round splat's kept region is a disc of radius sqrt(11.1 (a c - b^2)
    a / det) = sqrt(11.1 a): its candidate rectangle spans the tiles that
    disc's box meets, plus at most the growth margins."""
    f32 = np.float32
    a = np.array([4.0, 25.0, 100.0], f32)
    d = dict(a=a, b=np.zeros(3, f32), c=a.copy(), det=(a * a).astype(f32),
             px=np.array([100.3, 64.0, 130.7], f32), py=np.array([90.1, 64.0, 40.2], f32),
             x0=np.zeros(3, np.int64), x1=np.full(3, 20, np.int64),
             y0=np.zeros(3, np.int64), y1=np.full(3, 20, np.int64))
    d["tiles"] = np.full(3, 21 * 21, np.uint32)
    cand = fp.candidate_rect(d, 16, 16)
    r = np.sqrt(11.1 * a.astype(np.float64) / 0.9995)
    for i in range(3):
        lo = np.floor((d["px"][i] - r[i]) / 16.0)
        hi = np.floor((d["px"][i] + r[i]) / 16.0)
        assert cand["x0"][i] <= lo and cand["x1"][i] >= hi
        grown = r[i] * 1.001 * 1.001 + 0.06                   # the growth margins
        assert cand["x0"][i] >= np.floor((d["px"][i] - grown) / 16.0)
        assert cand["x1"][i] <= np.floor((d["px"][i] + grown) / 16.0)
