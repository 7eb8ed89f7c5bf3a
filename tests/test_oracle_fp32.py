"""Pins of the oracle's FP32 decision path against values fixed outside it:
published Philox vectors, libm in FP64, the Gumbel-max theorem."""
import math
import os

import numpy as np
import pytest

from oracle import fp32_path as fp

f32 = np.float32


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers(golden_dir):
    for r in _kat(golden_dir):
        out = fp.philox4x32_10(*r[:4], *r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_philox_vectorised_matches_scalar():
    i = np.arange(1000, dtype=np.uint32)
    vec = fp.philox4x32_10(i, 7, 0, 0, 123, 456)
    for j in (0, 1, 517, 999):
        sc = fp.philox4x32_10(j, 7, 0, 0, 123, 456)
        assert [int(v[j]) for v in vec] == [int(s) for s in sc]


def test_uniform24_exact_open_interval():
    x = np.array([0, 1, 511, 512, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = fp.uniform24(x)
    assert u.dtype == np.float32
    expect = [(2 * (int(v) >> 9) + 1) / 2.0 ** 24 for v in x]
    assert [float(a) for a in u] == expect           # exactly representable
    assert (u > 0).all() and (u < 1).all()


def _ulp_err(got, ref):
    got = np.asarray(got, np.float64)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    return np.abs(got - ref) / ulp


def test_log32_accuracy():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        np.exp(rng.uniform(np.log(2.0 ** -24), np.log(1.0), 200_000)),
        rng.uniform(1e-8, 30.0, 200_000),
        np.exp(rng.uniform(-80, 80, 100_000))]).astype(np.float32)
    x = x[x > 0]
    got = fp.log32(x)
    ref = np.log(x.astype(np.float64))
    nz = np.abs(ref) > 1e-3
    assert _ulp_err(got[nz], ref[nz]).max() <= 3.0
    # near x = 1 the absolute error is what matters
    assert np.abs(got[~nz] - ref[~nz]).max() <= 2e-10
    assert float(fp.log32(np.float32(1.0))) == 0.0
    assert float(fp.log32(np.float32(2.0))) == pytest.approx(math.log(2.0), rel=1e-7)


def test_exp32_accuracy():
    x = np.linspace(-80, 80, 400_001).astype(np.float32)
    got = fp.exp32(x)
    ref = np.exp(x.astype(np.float64))
    assert _ulp_err(got, ref).max() <= 2.0
    assert float(fp.exp32(np.float32(0.0))) == 1.0
    # clamp outside [-80, 80]
    assert float(fp.exp32(np.float32(200.0))) == float(fp.exp32(np.float32(80.0)))


def test_gumbel32_close_to_fp64():
    u0, _ = fp.gumbel_uniforms(100_000, 1, 2)
    g = fp.gumbel32(u0).astype(np.float64)
    ref = -np.log(-np.log(u0.astype(np.float64)))
    assert np.abs(g - ref).max() < 5e-6


def test_gumbel_max_frequency_is_sigmoid():
    """Gumbel-max theorem: P(l0 + g0 >= l1 + g1) = sigmoid(l0 - l1) (Sec. 3.3)."""
    n = 200_000
    for l0, l1 in [(0.0, 0.0), (1.5, -0.5), (-2.0, 0.3), (0.54, 0.0)]:
        logits = np.tile(np.array([[l0, l1]], np.float32), (n, 1))
        M, margin, _, _ = fp.sample_mask(logits, seed=99, it=5)
        p = 1.0 / (1.0 + math.exp(-(l0 - l1)))
        sd = math.sqrt(p * (1 - p) / n)
        assert abs(M.mean() - p) < 5 * sd, (l0, l1, M.mean(), p)
        assert ((margin >= 0) == (M == 1)).all()


def test_mask_index_zero_is_present():
    n = 10_000
    logits = np.zeros((n, 2), np.float32)
    logits[:, 0] = 30.0                      # overwhelmingly 'present'
    M, _, _, _ = fp.sample_mask(logits, 1, 0)
    assert M.all()
    logits[:, 0], logits[:, 1] = 0.0, 30.0
    M, _, _, _ = fp.sample_mask(logits, 1, 0)
    assert not M.any()


def test_mask_draws_depend_on_seed_and_iteration():
    l = np.zeros((50_000, 2), np.float32)
    a = fp.sample_mask(l, 1, 0)[0].astype(float)
    b = fp.sample_mask(l, 1, 1)[0].astype(float)
    c = fp.sample_mask(l, 2, 0)[0].astype(float)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.03
    assert abs(np.corrcoef(a, c)[0, 1]) < 0.03
    assert (fp.sample_mask(l, 1, 0)[0] == a).all()    # deterministic


def test_non_finite_inputs_are_culled():
    """NaN / inf means, NaN scales, a zero or NaN quaternion: the decision path
    culls the Gaussian (no tile), the others are untouched."""
    from paper_2412_20522_gb300 import scenes
    g, cams, _ = scenes.tiny_workload(500)
    ref = fp.project32(g.means, g.log_scales, g.quats, cams[0], 16, 16)
    m, s, q = g.means.copy(), g.log_scales.copy(), g.quats.copy()
    m[5] = np.nan
    m[9, 2] = np.inf
    s[17] = np.nan
    q[23] = 0.0
    q[31] = np.nan
    with np.errstate(invalid="ignore"):
        out = fp.project32(m, s, q, cams[0], 16, 16)
    bad = [5, 9, 17, 23, 31]
    assert (out["tiles"][bad] == 0).all() and (out["radius"][bad] == 0).all()
    good = np.setdiff1d(np.arange(500), bad)
    assert np.array_equal(out["tiles"][good], ref["tiles"][good])
