"""Oracle: the FP32 decision path (test infrastructure only).

Every integer the rasteriser derives from floating point -- the sampled mask
M_i (Sec. 3.3), the near-plane and determinant culls, the splat radius, the
tile rectangle that decides which 16x16 tiles a Gaussian intersects (Sec. 3.1)
and the depth key that orders the Gaussians of a pixel (Sec. 3.1, front to
back) -- is decided here in FP32, by a fixed sequence
of correctly rounded IEEE operations (add, sub, mul, div, sqrt, floor, ceil,
rint; never a fused multiply-add).  The CUDA kernels take the same decisions
with the same sequence, so the discrete outputs must agree bit for bit.

numpy float32 ufuncs are single correctly rounded IEEE operations, so each
line below is one rounding.  Transcendentals that feed a decision are the
project's own (``log32``, ``exp32``), built from textbook identities out of
those operations only, so the two sides cannot differ by a libm.

Numerical readings of points the paper leaves open (they come from the 3DGS
rasteriser the authors modified, Sec. 4.1 "Implementation Details"):
near plane 0.2, 0.3 low-pass added to the 2D covariance, Jacobian clamp at
1.3 tan(fov/2), radius ceil(3 sqrt(lambda_max)) with the eigenvalue gap floored
at 0.1, tile rectangle = tiles overlapped by the square [p +- r].  The 2D
covariance is formed from its factor P = J W R S (Sigma_bar = P P^T + 0.3 I),
its determinant by Cauchy-Binet and its eigenvalue gap as a sum of squares, so
that no decision rests on a cancellation.
"""
from __future__ import annotations

import numpy as np

f32 = np.float32
u32 = np.uint32

# constants as exact float32 bit patterns (hex floats)
C_INV3 = f32(float.fromhex("0x1.555556p-2"))
C_INV5 = f32(float.fromhex("0x1.99999ap-3"))
C_INV7 = f32(float.fromhex("0x1.24924ap-3"))
C_INV9 = f32(float.fromhex("0x1.c71c72p-4"))
C_INV11 = f32(float.fromhex("0x1.745d18p-4"))
LN2_HI = f32(float.fromhex("0x1.62e4p-1"))
LN2_LO = f32(float.fromhex("0x1.7f7d1cp-20"))
INV_LN2 = f32(float.fromhex("0x1.715476p+0"))
SQRT2 = f32(float.fromhex("0x1.6a09e6p+0"))
INV_FACT = [f32(1.0), f32(1.0), f32(0.5),
            f32(float.fromhex("0x1.555556p-3")), f32(float.fromhex("0x1.555556p-5")),
            f32(float.fromhex("0x1.111112p-7")), f32(float.fromhex("0x1.6c16c2p-10")),
            f32(float.fromhex("0x1.a01a02p-13"))]
LOWPASS = f32(0.3)
ALPHA_MIN = f32(1.0) / f32(255.0)


# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
# as 1, 2, 3", SC'11).  Written from the published round function.
# ---------------------------------------------------------------------------
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32 with 10 rounds; all arguments uint32 (arrays ok)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64)
    k1 = np.asarray(k1, dtype=np.uint64)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(PHILOX_W0)) & mask
            k1 = (k1 + np.uint64(PHILOX_W1)) & mask
        p0 = c0 * np.uint64(PHILOX_M0)
        p1 = c2 * np.uint64(PHILOX_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def uniform24(x):
    """u = (2*(x>>9)+1) * 2^-24: an exactly representable float32 in (0, 1)."""
    v = ((np.asarray(x, dtype=np.uint32) >> u32(9)) << u32(1)) | u32(1)
    return v.astype(np.float32) * f32(2.0 ** -24)


# ---------------------------------------------------------------------------
# Own FP32 log and exp, from textbook identities (no libm).
# ---------------------------------------------------------------------------

def log32(x):
    """log(x) for positive normal float32 x.

    x = m 2^e with m in [1/sqrt2, sqrt2); log m = 2 atanh(s), s = (m-1)/(m+1),
    atanh(s) = s (1 + s^2/3 + s^4/5 + ... + s^10/11)  (|s| <= 0.1716);
    log x = e ln2_hi + (e ln2_lo + log m)  (Cody-Waite split of ln 2).
    """
    x = np.asarray(x, dtype=np.float32)
    bits = x.view(np.uint32)
    e = ((bits >> u32(23)) & u32(0xFF)).astype(np.int32) - 127
    m = ((bits & u32(0x7FFFFF)) | u32(0x3F800000)).view(np.float32)
    big = m >= SQRT2
    m = np.where(big, m * f32(0.5), m).astype(np.float32)
    e = e + big.astype(np.int32)
    s = (m - f32(1.0)) / (m + f32(1.0))
    z = s * s
    p = C_INV11
    for c in (C_INV9, C_INV7, C_INV5, C_INV3, f32(1.0)):
        p = p * z
        p = p + c
    lm = (s * f32(2.0)) * p
    ef = e.astype(np.float32)
    return (ef * LN2_HI + (ef * LN2_LO + lm)).astype(np.float32)


def exp32(x):
    """exp(x) for float32 x, input clamped to [-80, 80] (by comparisons, so
    a NaN stays NaN and the Gaussian is culled downstream).

    Cody-Waite reduction x = k ln2 + r, k = rint(x / ln2), |r| <= ln2/2,
    exp(r) by its Taylor series to r^7/7! in Horner form, then scaled by 2^k
    (built exactly from the exponent bits).
    """
    x = np.asarray(x, dtype=np.float32)
    x = np.where(x < f32(-80.0), f32(-80.0), np.where(x > f32(80.0), f32(80.0), x))
    nan = np.isnan(x)
    k = np.rint(np.where(nan, f32(0.0), x) * INV_LN2).astype(np.float32)
    r = (x - k * LN2_HI) - k * LN2_LO
    p = INV_FACT[7]
    for j in range(6, -1, -1):
        p = p * r
        p = p + INV_FACT[j]
    ki = k.astype(np.int32)
    two_k = ((ki + 127).astype(np.uint32) << u32(23)).view(np.float32)
    return np.where(nan, np.float32(np.nan), p * two_k).astype(np.float32)


# ---------------------------------------------------------------------------
# Mask sample (Sec. 3.3): Gumbel-max over the two existence scores.
# ---------------------------------------------------------------------------

def gumbel_uniforms(n, seed, it, index_offset=0, draw=0):
    """The two uniforms u_0, u_1 of Gaussian i: Philox4x32-10 with
    counter (i, iter_lo, iter_hi, draw) and key (seed_lo, seed_hi); i counts
    from ``index_offset`` (the Gaussian's index in a batch of scenes).  The
    training sample is draw 0; the pruning draws are 1, 2, ..."""
    i = (np.arange(n, dtype=np.uint64) + np.uint64(index_offset)).astype(np.uint32)
    it = int(it)
    seed = int(seed)
    x = philox4x32_10(i, np.full(n, it & 0xFFFFFFFF, np.uint32),
                      np.full(n, (it >> 32) & 0xFFFFFFFF, np.uint32),
                      np.full(n, int(draw) & 0xFFFFFFFF, np.uint32),
                      seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return uniform24(x[0]), uniform24(x[1])


def gumbel32(u):
    """g = -log(-log u) in FP32 with the own log."""
    return -log32(-log32(u))


def sample_mask(mask_logits, seed, it, index_offset=0, draw=0):
    """Hard Gumbel-max sample M_i = [l_0 + g_0 >= l_1 + g_1] (index 0 = present,
    ties to 'present'), decided in FP32.  Returns (M uint8, margin f32, u0, u1)."""
    l = np.asarray(mask_logits, dtype=np.float32)
    u0, u1 = gumbel_uniforms(l.shape[0], seed, it, index_offset, draw)
    a0 = l[:, 0] + gumbel32(u0)
    a1 = l[:, 1] + gumbel32(u1)
    d = a0 - a1
    return (d >= f32(0.0)).astype(np.uint8), d, u0, u1


def ste_mask(mask_logits, ste_logit):
    """Deterministic threshold mask of the straight-through ablation (Sec. 4.3,
    "Effect of Gumbel Softmax"): M_i = [sigmoid(l_0 - l_1) > theta], decided
    as l_0 - l_1 > logit(theta) (sigmoid is increasing), one FP32 subtraction
    and one comparison.  Returns (M uint8, d = l_0 - l_1 f32)."""
    l = np.asarray(mask_logits, dtype=np.float32)
    d = l[:, 0] - l[:, 1]
    return (d > f32(ste_logit)).astype(np.uint8), d


def prune_keep(mask_logits, seed, it, n_draws=10, index_offset=0):
    """Pruning rule of Sec. 3.5: sample every Gaussian n_draws times (draws
    1..n_draws of the noise stream) and keep those sampled present at least
    once.  Returns keep (uint8)."""
    l = np.asarray(mask_logits, dtype=np.float32)
    keep = np.zeros(l.shape[0], np.uint8)
    for d in range(1, int(n_draws) + 1):
        M, _, _, _ = sample_mask(l, seed, it, index_offset, draw=d)
        keep |= M
    return keep


# ---------------------------------------------------------------------------
# Projection, covariance, radius, tile rectangle (Sec. 3.1).
# ---------------------------------------------------------------------------

def quat_to_rot32(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z), FP32.
    Returns (R [N,3,3], valid) ; a zero quaternion is invalid."""
    q = np.asarray(q, dtype=np.float32)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    n2 = ((w * w + x * x) + y * y) + z * z
    valid = n2 > f32(0.0)
    nrm = np.sqrt(np.where(valid, n2, f32(1.0)))
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    two, one = f32(2.0), f32(1.0)
    R = np.empty((q.shape[0], 3, 3), np.float32)
    R[:, 0, 0] = one - two * (y * y + z * z)
    R[:, 0, 1] = two * (x * y - w * z)
    R[:, 0, 2] = two * (x * z + w * y)
    R[:, 1, 0] = two * (x * y + w * z)
    R[:, 1, 1] = one - two * (x * x + z * z)
    R[:, 1, 2] = two * (y * z - w * x)
    R[:, 2, 0] = two * (x * z - w * y)
    R[:, 2, 1] = two * (y * z + w * x)
    R[:, 2, 2] = one - two * (x * x + y * y)
    return R, valid


def project32(means, log_scales, quats, cam, tile_w=16, tile_h=16):
    """The FP32 decision path for one camera.

    Returns a dict with, per Gaussian: tz (depth), px, py (2D mean, pixels),
    a, b, c of the low-passed 2D covariance [[a, b], [b, c]], its determinant
    det, disc = ((a-c)/2)^2 + b^2, radius (int32),
    rect x0, y0, x1, y1 (inclusive tile bounds), tiles (tiles touched, uint32)
    and depth_bits (uint32 of tz).
    """
    p = np.asarray(means, dtype=np.float32)
    V = np.asarray(cam.viewmat, dtype=np.float32)
    fx, fy = f32(cam.fx), f32(cam.fy)
    cx, cy = f32(cam.cx), f32(cam.cy)
    W, H = cam.width, cam.height
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    t = [((V[r, 0] * x + V[r, 1] * y) + V[r, 2] * z) + V[r, 3] for r in range(3)]
    tx, ty, tz = t
    in_front = tz > f32(cam.near)
    tzs = np.where(in_front, tz, f32(1.0))           # keep the arithmetic finite
    ux = tx / tzs
    uy = ty / tzs
    px = fx * ux + cx
    py = fy * uy + cy

    # Sigma_bar = P P^T + lowpass I with P = J W R S  (2x3): the same matrix as
    # J W Sigma W^T J^T + lowpass I, formed from its factor so that the
    # determinant (Cauchy-Binet) and the eigenvalue gap are sums of squares.
    s = exp32(log_scales)
    R, qvalid = quat_to_rot32(quats)
    M = R * s[:, None, :]                      # M = R S (columns scaled)

    # Jacobian of the perspective map at the clamped point
    tanx = (f32(W) * f32(0.5)) / fx
    tany = (f32(H) * f32(0.5)) / fy
    limx = f32(1.3) * tanx
    limy = f32(1.3) * tany
    txc = np.minimum(limx, np.maximum(-limx, ux)) * tzs
    tyc = np.minimum(limy, np.maximum(-limy, uy)) * tzs
    tz2 = tzs * tzs
    j00 = fx / tzs
    j02 = -((fx * txc) / tz2)
    j11 = fy / tzs
    j12 = -((fy * tyc) / tz2)
    # T = J W (W = rotation part of the view matrix); J has zeros at (0,1), (1,0)
    T0 = [j00 * V[0, k] + j02 * V[2, k] for k in range(3)]
    T1 = [j11 * V[1, k] + j12 * V[2, k] for k in range(3)]
    # P = T M
    P0 = [(T0[0] * M[:, 0, k] + T0[1] * M[:, 1, k]) + T0[2] * M[:, 2, k] for k in range(3)]
    P1 = [(T1[0] * M[:, 0, k] + T1[1] * M[:, 1, k]) + T1[2] * M[:, 2, k] for k in range(3)]
    n0 = (P0[0] * P0[0] + P0[1] * P0[1]) + P0[2] * P0[2]
    n1 = (P1[0] * P1[0] + P1[1] * P1[1]) + P1[2] * P1[2]
    a = n0 + LOWPASS
    b = (P0[0] * P1[0] + P0[1] * P1[1]) + P0[2] * P1[2]
    c = n1 + LOWPASS
    m01 = P0[0] * P1[1] - P0[1] * P1[0]
    m02 = P0[0] * P1[2] - P0[2] * P1[0]
    m12 = P0[1] * P1[2] - P0[2] * P1[1]
    det = (((m01 * m01 + m02 * m02) + m12 * m12) + LOWPASS * (n0 + n1)) + LOWPASS * LOWPASS
    mid = f32(0.5) * (a + c)
    hd = f32(0.5) * (a - c)
    disc = hd * hd + b * b
    lam = mid + np.sqrt(np.maximum(f32(0.1), disc))
    rf = np.ceil(f32(3.0) * np.sqrt(lam))
    ok = in_front & qvalid & (det > f32(0.0)) & np.isfinite(px) & np.isfinite(py) & np.isfinite(rf)
    # radius capped at 1e9 px (exact in float32 and in int32)
    rf = np.where(ok, np.minimum(rf, f32(1e9)), f32(0.0)).astype(np.float32)

    gx = (W + tile_w - 1) // tile_w
    gy = (H + tile_h - 1) // tile_h
    twf, thf = f32(tile_w), f32(tile_h)
    x0 = np.maximum(np.floor((px - rf) / twf), f32(0.0))
    x1 = np.minimum(np.floor((px + rf) / twf), f32(gx - 1))
    y0 = np.maximum(np.floor((py - rf) / thf), f32(0.0))
    y1 = np.minimum(np.floor((py + rf) / thf), f32(gy - 1))
    nonempty = ok & (rf > f32(0.0)) & (x0 <= x1) & (y0 <= y1)
    x0i = np.where(nonempty, x0, 0).astype(np.int64)
    x1i = np.where(nonempty, x1, -1).astype(np.int64)
    y0i = np.where(nonempty, y0, 0).astype(np.int64)
    y1i = np.where(nonempty, y1, -1).astype(np.int64)
    tiles = ((x1i - x0i + 1) * (y1i - y0i + 1)).astype(np.uint32)
    radius = np.where(nonempty, rf, f32(0.0)).astype(np.int32)
    return dict(tz=tz, px=px, py=py, a=a, b=b, c=c, det=det, disc=disc, radius=radius,
                x0=x0i, x1=x1i, y0=y0i, y1=y1i, tiles=tiles,
                depth_bits=tz.view(np.uint32).copy(), visible=nonempty,
                grid=(gx, gy))


# ---------------------------------------------------------------------------
# Tile filter of the binning: a Gaussian is kept in a tile of its rectangle
# unless, at every pixel centre of the tile, its quadratic form
# q = d^T Sigma_bar^-1 d exceeds 2 ln 255 -- where alpha = o exp(-q/2) <
# 1/255 for any opacity o <= 1, so the Gaussian is filtered at every pixel
# of the tile (Sec. 3.1: only Gaussians with alpha above the floor take
# part).  Dropping such pairs changes no image and no gradient; it shortens
# the tile lists.  The test takes the minimum of the numerator
# N = c dx^2 - 2 b dx dy + a dy^2 = det q over the box of pixel centres (the
# centre inside, else the minimum of each edge at its clamped stationary
# point) and keeps the pair if N <= 11.1 det + 1e-4 (|terms| summed): 11.1 >
# 2 ln 255 = 11.0825, and the relative slack covers the rounding of N.
# ---------------------------------------------------------------------------
T_BIN = f32(11.1)
REL_BIN = f32(1e-4)


# ---------------------------------------------------------------------------
# Candidate rectangle of the filtered binning.  A tile the filter keeps holds
# a point d (pixel-centre offset from the mean) with computed
# N <= 11.1 det + 1e-4 S, S = t1 + |2 t2| + t3.  N's rounding moves it by at
# most 4 eps S (eps = 2^-24), and S <= 2 (c dx^2 + a dy^2) because b^2 < a c;
# so every kept point satisfies d^T M d <= T with
# M = [[c (1 - 2k), -b], [-b, a (1 - 2k)]], k = 1.0025e-4, T = 11.1 det
# (1 + 1e-7).  With kappa = 0.9995 <= (1 - 2k)^2 the ellipse d^T M' d <= T,
# M' = [[c sqrt(kappa), -b], [-b, a sqrt(kappa)]], contains it, and its
# bounding box has half-widths sqrt(T a sqrt(kappa) / det') <=
# sqrt(T a / det'), det' = kappa a c - b^2 (likewise y with c).  Evaluated in
# correctly rounded FP32 in this order: det' only where it is at least 1e-3
# a c (there its rounding error is below 2e-4 of it), the half-widths grown by
# 1e-3 relative and 0.05 px (the rounding of det', of the filter's offsets and
# of px -+ h), the box holds every kept tile: the candidates are the tiles of
# the 3-sigma square that meet it.  Elsewhere the square stays.
# ---------------------------------------------------------------------------
CAND_KAPPA = f32(0.9995)
CAND_MIN_DET = f32(1e-3)
CAND_GROW = f32(1.001)
CAND_MARGIN = f32(0.05)


def candidate_rect(fp, tile_w=16, tile_h=16):
    """The tiles of each Gaussian's 3-sigma rectangle that the tile filter can
    keep: dict x0, x1, y0, y1 (inclusive, int64) and tiles (uint32); a
    Gaussian with none gets tiles 0."""
    vis = fp["tiles"] > 0
    one = f32(1.0)
    a = np.where(vis, fp["a"], one)
    b = np.where(vis, fp["b"], f32(0.0))
    c = np.where(vis, fp["c"], one)
    tdet = T_BIN * np.where(vis, fp["det"], one)
    px = np.where(vis, fp["px"], f32(0.0))
    py = np.where(vis, fp["py"], f32(0.0))
    with np.errstate(all="ignore"):
        ac = a * c
        detk = CAND_KAPPA * ac - b * b
        tight = vis & (detk > CAND_MIN_DET * ac)
        T = tdet * CAND_GROW
        dk = np.where(tight, detk, one)
        hx = np.sqrt((T * a) / dk) * CAND_GROW + CAND_MARGIN
        hy = np.sqrt((T * c) / dk) * CAND_GROW + CAND_MARGIN
        lx = np.floor((px - hx) / f32(tile_w))
        ux = np.floor((px + hx) / f32(tile_w))
        ly = np.floor((py - hy) / f32(tile_h))
        uy = np.floor((py + hy) / f32(tile_h))
    x0, x1, y0, y1 = (fp[k].astype(np.float64) for k in ("x0", "x1", "y0", "y1"))
    x0 = np.where(tight, np.maximum(x0, lx.astype(np.float64)), x0)
    x1 = np.where(tight, np.minimum(x1, ux.astype(np.float64)), x1)
    y0 = np.where(tight, np.maximum(y0, ly.astype(np.float64)), y0)
    y1 = np.where(tight, np.minimum(y1, uy.astype(np.float64)), y1)
    ok = vis & (x0 <= x1) & (y0 <= y1)
    x0i = np.where(ok, x0, 0).astype(np.int64)
    x1i = np.where(ok, x1, -1).astype(np.int64)
    y0i = np.where(ok, y0, 0).astype(np.int64)
    y1i = np.where(ok, y1, -1).astype(np.int64)
    tiles = ((x1i - x0i + 1) * (y1i - y0i + 1)).astype(np.uint32)
    return dict(x0=x0i, x1=x1i, y0=y0i, y1=y1i, tiles=tiles)


def tile_filter_params(fp):
    """Per Gaussian: (t det, b / a, b / c), correctly rounded FP32."""
    a, b, c, det = fp["a"], fp["b"], fp["c"], fp["det"]
    ok = fp["tiles"] > 0
    one = f32(1.0)
    aa = np.where(ok, a, one)
    cc = np.where(ok, c, one)
    return T_BIN * det, b / aa, b / cc


def _edge_hit(N_terms, tdet):
    t1, t2, t3 = N_terms
    t22 = t2 + t2
    N = (t1 - t22) + t3
    bnd = (t1 + np.abs(t22)) + t3
    return N <= tdet + REL_BIN * bnd


def tile_hit(px, py, a, b, c, tdet, rba, rbc, tx, ty, tile_w, tile_h):
    """Keep (True) or drop the Gaussian/tile pairs given per pair (arrays of
    equal length; tile column tx and row ty within the view)."""
    X0 = (tx * tile_w).astype(np.float32) + f32(0.5)
    Y0 = (ty * tile_h).astype(np.float32) + f32(0.5)
    X1 = X0 + f32(tile_w - 1)
    Y1 = Y0 + f32(tile_h - 1)
    dx0, dx1 = X0 - px, X1 - px
    dy0, dy1 = Y0 - py, Y1 - py
    hit = (dx0 <= f32(0.0)) & (dx1 >= f32(0.0)) & (dy0 <= f32(0.0)) & (dy1 >= f32(0.0))
    for dxe in (dx0, dx1):                      # vertical edges
        dyc = np.minimum(np.maximum(rba * dxe, dy0), dy1)
        hit |= _edge_hit((c * (dxe * dxe), (b * dxe) * dyc, a * (dyc * dyc)), tdet)
    for dye in (dy0, dy1):                      # horizontal edges
        dxc = np.minimum(np.maximum(rbc * dye, dx0), dx1)
        hit |= _edge_hit((c * (dxc * dxc), (b * dxc) * dye, a * (dye * dye)), tdet)
    return hit
