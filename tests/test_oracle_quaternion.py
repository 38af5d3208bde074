"""Pins of the QSSIM oracle (oracle/quaternion.py, Section "Quaternion SSIM").

The quaternion algebra is checked against its defining relations; the score
against closed forms that do not go through the Hamilton product: identity,
constant colours (vector dot and cross products), grey pictures (the global
grayscale SSIM of sqrt(3) times the grey level, written out with scalars and
the section's (M-1)(N-1) normalisation) and a hue rotation about the grey
axis, whose correlation has both a real and a vector part.
"""
import numpy as np
import pytest

from oracle import constants
from oracle import quaternion as Q

ONE, I, J, K = np.eye(4)


def test_hamilton_product_defining_relations():
    for u in (I, J, K):
        np.testing.assert_array_equal(Q.qmul(u, u), -ONE)
    np.testing.assert_array_equal(Q.qmul(Q.qmul(I, J), K), -ONE)
    np.testing.assert_array_equal(Q.qmul(I, J), K)
    np.testing.assert_array_equal(Q.qmul(J, K), I)
    np.testing.assert_array_equal(Q.qmul(K, I), J)
    np.testing.assert_array_equal(Q.qmul(J, I), -K)
    r = np.random.default_rng(5)
    p, q, s = r.normal(size=(3, 7, 4))
    np.testing.assert_allclose(Q.qmul(Q.qmul(p, q), s), Q.qmul(p, Q.qmul(q, s)), atol=1e-12)
    np.testing.assert_allclose(Q.qabs(Q.qmul(p, q)), Q.qabs(p) * Q.qabs(q), rtol=1e-13)
    np.testing.assert_allclose(Q.qconj(Q.qmul(p, q)), Q.qmul(Q.qconj(q), Q.qconj(p)), atol=1e-12)
    # pure quaternions: a conj(b) = a.b - a x b
    a, b = p[:, 1:], q[:, 1:]
    pa, pb = Q.to_quaternion(a[:, 0], a[:, 1], a[:, 2]), Q.to_quaternion(b[:, 0], b[:, 1], b[:, 2])
    got = Q.qmul(pa, Q.qconj(pb))
    np.testing.assert_allclose(got[:, 0], np.sum(a * b, axis=1), atol=1e-12)
    np.testing.assert_allclose(got[:, 1:], -np.cross(a, b), atol=1e-12)


def _picture(seed, shape=(9, 14), lo=0.0, hi=255.0):
    r = np.random.default_rng(seed)
    return tuple(np.round(r.uniform(lo, hi, shape)) for _ in range(3))


def test_identity_gives_one():
    x = _picture(1)
    for K1, K2 in ((0.01, 0.03), (0.0, 0.0)):
        lum, cs, s = Q.qssim_terms(x, x, K1, K2)
        assert lum == pytest.approx(1.0, abs=1e-15)
        assert cs == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("a,b", [((200.0, 10.0, 40.0), (180.0, 30.0, 45.0)), ((10.0, 20.0, 30.0), (30.0, 10.0, 20.0)),
                                 ((0.0, 0.0, 0.0), (50.0, 60.0, 70.0))])
def test_constant_colours_give_the_dc_term(a, b):
    """Constant pictures: no AC, so the contrast factor is C2 / C2 = 1 and the
    score is |2 a conj(b) + C1| / (|a|^2 + |b|^2 + C1), whose modulus is
    sqrt((2 a.b + C1)^2 + 4 |a x b|^2)."""
    shape = (5, 6)
    x = tuple(np.full(shape, v) for v in a)
    y = tuple(np.full(shape, v) for v in b)
    C1, _ = constants()
    av, bv = np.array(a), np.array(b)
    want = np.sqrt((2 * av @ bv + C1) ** 2 + 4 * np.sum(np.cross(av, bv) ** 2)) / (av @ av + bv @ bv + C1)
    lum, cs, s = Q.qssim_terms(x, y)
    assert cs == pytest.approx(1.0, abs=1e-15)
    assert lum == pytest.approx(want, rel=1e-14)
    assert s == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_grey_pictures_reduce_to_grayscale_ssim_of_sqrt3_v(sign):
    """r = g = b = v: q = v (i + j + k), so every quaternion is parallel to
    the grey axis, the cross products vanish and QSSIM is the modulus of the
    global grayscale SSIM of sqrt(3) v (same C1, C2 and normalisation)."""
    r = np.random.default_rng(2)
    shape = (12, 17)
    v = np.round(r.uniform(20, 230, shape))
    w = np.clip(np.round(128 + sign * (v - 128) + r.normal(0, 9, shape)), 0, 255)
    x, y = np.sqrt(3.0) * v, np.sqrt(3.0) * w
    M, N = shape
    C1, C2 = constants()
    mx, my = x.mean(), y.mean()
    vx = np.sum((x - mx) ** 2) / ((M - 1) * (N - 1))
    vy = np.sum((y - my) ** 2) / ((M - 1) * (N - 1))
    cxy = np.sum((x - mx) * (y - my)) / ((M - 1) * (N - 1))
    want = abs((2 * mx * my + C1) / (mx ** 2 + my ** 2 + C1) * (2 * cxy + C2) / (vx + vy + C2))
    got = Q.qssim((v, v, v), (w, w, w))
    assert got == pytest.approx(want, rel=1e-13)
    if sign < 0:
        assert cxy < 0  # anti-correlated: the modulus folds the sign


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.2, np.pi / 2, 2.5])
def test_hue_rotation_about_grey_axis(theta):
    """Reference = a constant colour m plus a checkerboard of +a / -a with a
    perpendicular to the grey axis n; distorted = m plus the same pattern of
    R a, R the rotation by theta about n.  Then |ac| is unchanged, and
    sigma_{ref,dis} = V (cos theta - sin theta n) with V = (M N |a|^2) /
    ((M-1)(N-1)), so the contrast factor is
    sqrt(4 V^2 + 4 V C2 cos theta + C2^2) / (2 V + C2)."""
    M, N = 6, 8
    n = np.ones(3) / np.sqrt(3.0)
    a = np.array([12.0, -7.0, -5.0])  # a . n = 0
    Ra = np.cos(theta) * a + np.sin(theta) * np.cross(n, a)  # Rodrigues, a perpendicular to n
    m = np.array([120.0, 100.0, 90.0])
    s = np.where((np.add.outer(np.arange(M), np.arange(N)) % 2) == 0, 1.0, -1.0)
    x = tuple(m[c] + s * a[c] for c in range(3))
    y = tuple(m[c] + s * Ra[c] for c in range(3))
    C1, C2 = constants()
    V = M * N * (a @ a) / ((M - 1) * (N - 1))
    want_cs = np.sqrt(4 * V * V + 4 * V * C2 * np.cos(theta) + C2 * C2) / (2 * V + C2)
    lum, cs, _ = Q.qssim_terms(x, y)
    assert lum == pytest.approx(1.0, abs=1e-15)  # same mean colour
    assert cs == pytest.approx(want_cs, rel=1e-13)


def test_rejects_too_small_or_mismatched():
    x = _picture(3, (1, 5))
    with pytest.raises(ValueError):
        Q.qssim(x, x)
    with pytest.raises(ValueError):
        Q.qssim(_picture(3, (4, 5)), _picture(3, (5, 4)))
