"""Pins of the scale oracle (oracle/scales.py): the automatic downscaling
factor against the paper's examples, block-mean downscaling against the 2x2
pyramid and reshape means, and the 9/7 wavelet low-pass against its defining
properties (unit DC gain, symmetry, exact on linear ramps away from the
border)."""
import numpy as np
import pytest

import oracle
from oracle import scales as S


def test_downscale_factor_rules():
    assert S.downscale_factor(1080, 1920) == 4          # round(1080 / 256 = 4.22)
    assert S.downscale_factor(200, 300) == 1
    assert S.downscale_factor(384, 1000) == 2           # 1.5 rounds up
    assert S.downscale_factor(383, 1000) == 1
    # the paper's example of the ceil rule's jump: H = 510 -> 2, H = 520 -> 3
    assert S.downscale_factor(510, 900, "ceil_h") == 2
    assert S.downscale_factor(520, 900, "ceil_h") == 3
    assert S.downscale_factor(100, 900, "ceil_h") == 1
    with pytest.raises(ValueError):
        S.downscale_factor(10, 10, "nearest")


def test_block_mean():
    r = np.random.default_rng(0)
    a = r.uniform(0, 255, (23, 31))
    np.testing.assert_array_equal(S.downscale_block(a, 2), oracle.downsample2x2(a))
    np.testing.assert_array_equal(S.downscale_block(a, 1), a)
    b = S.downscale_block(a, 3)
    assert b.shape == (7, 10)
    np.testing.assert_allclose(b, a[:21, :30].reshape(7, 3, 10, 3).mean(axis=(1, 3)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(S.downscale_block(np.full((9, 9), 7.0), 4), 7.0)


def test_cdf97_lowpass_properties():
    h = S.CDF97_LOWPASS
    assert h.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_array_equal(h, h[::-1])                       # symmetric
    t = np.arange(-4, 5)
    assert (h * t).sum() == pytest.approx(0.0, abs=1e-15)           # no shift of a linear ramp
    assert h[4] == pytest.approx(0.602949018236, abs=1e-12)         # the published centre tap, normalised


def test_pyramid_97_constant_linear_and_transpose():
    np.testing.assert_allclose(S.pyramid_97(np.full((20, 26), 3.5)), 3.5, rtol=0, atol=1e-13)
    i, j = np.mgrid[0:40, 0:46]
    ramp = 3.0 * i - 2.0 * j + 5.0
    out = S.pyramid_97(ramp)
    assert out.shape == (20, 23)
    oi, oj = np.mgrid[0:20, 0:23]
    inner = (oi >= 2) & (oi <= 17) & (oj >= 2) & (oj <= 20)        # windows clear of the border
    np.testing.assert_allclose(out[inner], (3.0 * 2 * oi - 2.0 * 2 * oj + 5.0)[inner], rtol=0, atol=1e-11)
    r = np.random.default_rng(1)
    a = r.uniform(0, 1, (17, 30))
    np.testing.assert_allclose(S.pyramid_97(a.T), S.pyramid_97(a).T, rtol=0, atol=1e-14)


def test_symmetric_extension_border():
    # a row that rises by one per sample reflects at the border: output 0
    # centred on sample 0 sees samples 4 3 2 1 0 1 2 3 4 -> sum h_t |t|
    a = np.tile(np.arange(12.0), (4, 1))
    out = S.pyramid_97(a)
    ref = (S.CDF97_LOWPASS * np.abs(np.arange(-4, 5))).sum()
    assert out[0, 0] == pytest.approx(ref, abs=1e-13)


def test_msssim_97_pyramid_identity():
    r = np.random.default_rng(2)
    x = r.integers(0, 256, (180, 200)).astype(np.uint8)
    s, per = oracle.msssim(x, x, pyramid="97")
    assert s == pytest.approx(1.0, abs=1e-12)
    assert len(per) == 5


def test_rgb_to_ycbcr():
    v = np.linspace(0, 255, 12).reshape(3, 4)
    y, cb, cr = S.rgb_to_ycbcr(v, v, v)          # grey: the luma weights sum to one
    np.testing.assert_allclose(y, v, rtol=0, atol=1e-12)
    np.testing.assert_allclose(cb, 0.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(cr, 0.0, rtol=0, atol=1e-12)
    z = np.zeros((2, 2))
    y, cb, cr = S.rgb_to_ycbcr(z + 100, z, z)    # pure red
    np.testing.assert_allclose(y, 21.3)
    np.testing.assert_allclose(cb, 0.539 * -21.3)
    np.testing.assert_allclose(cr, 0.635 * (100 - 21.3))
    y, cb, cr = S.rgb_to_ycbcr(z, z, z + 100)    # pure blue
    np.testing.assert_allclose(cb, 0.539 * (100 - 7.2))
