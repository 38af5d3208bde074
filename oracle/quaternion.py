"""FP64 oracle of QSSIM (Section "Quaternion SSIM" of arXiv 2101.06354).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.  Pinned by
``tests/test_oracle_quaternion.py``.

The section writes each colour pixel as the pure quaternion
q(m, n) = r i + g j + b k, splits the picture into its mean ("DC") mu_q and
the deviations ("AC") ac_q = q - mu_q, defines a quaternion contrast sigma_q
and a quaternion correlation sigma_{q_ref,dis} (the mean of ac_ref times the
conjugate of ac_dis), and combines them like the grayscale SSIM.  All sums run
over the whole M x N picture: one score per picture.

The printed formula is garbled in three places; the readings taken here:
  * sigma_q: the printed root of the mean of the unsquared norm ||ac_q||_2 is
    read as the root of the mean of the squared norm |ac_q|^2 (a variance,
    and the only reading for which sigma_{q,q} = sigma_q^2);
  * the squares mu^2 and sigma^2 in the denominators are squared moduli
    |mu|^2, sigma^2 (for a pure quaternion mu, mu mu = -|mu|^2);
  * the second factor divides by sigma_ref^2 + sigma_dis^2 (the printed
    mu_ref^2 + mu_dis^2 repeats the first denominator) and carries the factor
    2 of the grayscale cs term, so that QSSIM(x, x) = 1;
  * the stabilising constants C1 = (K1 L)^2, C2 = (K2 L)^2 of the grayscale
    formula are added to numerator and denominator of the two factors
    (K1 = K2 = 0 gives the printed constant-free form);
  * the normalisation 1/((M-1)(N-1)) of sigma_q and sigma_{q_ref,dis} is
    taken as printed (M, N >= 2).
So, with |.| the quaternion modulus,

    QSSIM = | (2 mu_ref conj(mu_dis) + C1) / (|mu_ref|^2 + |mu_dis|^2 + C1) |
          * | (2 sigma_{ref,dis} + C2) / (sigma_ref^2 + sigma_dis^2 + C2) |.
"""
from __future__ import annotations

import numpy as np

from . import constants


def qmul(p, q):
    """Hamilton product of quaternions stored as (..., 4) arrays
    (w, x, y, z) = w + x i + y j + z k."""
    p, q = np.asarray(p, np.float64), np.asarray(q, np.float64)
    a1, b1, c1, d1 = np.moveaxis(p, -1, 0)
    a2, b2, c2, d2 = np.moveaxis(q, -1, 0)
    return np.stack([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2,
                     a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                     a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2,
                     a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2], axis=-1)


def qconj(q):
    """Quaternion conjugate: w - x i - y j - z k."""
    q = np.asarray(q, np.float64)
    return q * np.array([1.0, -1.0, -1.0, -1.0])


def qabs(q) -> np.ndarray:
    """Quaternion modulus sqrt(w^2 + x^2 + y^2 + z^2)."""
    return np.sqrt(np.sum(np.asarray(q, np.float64) ** 2, axis=-1))


def to_quaternion(r, g, b) -> np.ndarray:
    """The pure quaternion picture q = r i + g j + b k, shape (M, N, 4)."""
    r, g, b = (np.asarray(c, np.float64) for c in (r, g, b))
    return np.stack([np.zeros_like(r), r, g, b], axis=-1)


def qssim_terms(tri_ref, tri_dis, K1: float = 0.01, K2: float = 0.03, L: float = 255.0):
    """The two factors of QSSIM for one picture pair (each a tuple of three
    planes of the same M x N shape, M, N >= 2): returns (l, cs, qssim) with
    l = |2 mu_ref conj(mu_dis) + C1| / (|mu_ref|^2 + |mu_dis|^2 + C1),
    cs = |2 sigma_{ref,dis} + C2| / (sigma_ref^2 + sigma_dis^2 + C2) and
    qssim = l * cs."""
    qr, qd = to_quaternion(*tri_ref), to_quaternion(*tri_dis)
    M, N = qr.shape[:2]
    if qd.shape != qr.shape or M < 2 or N < 2:
        raise ValueError("need two pictures of one shape, at least 2 x 2")
    C1, C2 = constants(K1, K2, L)
    norm = 1.0 / ((M - 1) * (N - 1))
    # DC: the mean quaternion; AC: the deviations from it
    mu_r = qr.reshape(-1, 4).sum(axis=0) / (M * N)
    mu_d = qd.reshape(-1, 4).sum(axis=0) / (M * N)
    ac_r, ac_d = qr - mu_r, qd - mu_d
    # contrast (squared-norm reading) and quaternion correlation
    var_r = norm * np.sum(qabs(ac_r) ** 2)
    var_d = norm * np.sum(qabs(ac_d) ** 2)
    cor = norm * qmul(ac_r, qconj(ac_d)).reshape(-1, 4).sum(axis=0)
    one = np.array([1.0, 0.0, 0.0, 0.0])
    lum = qabs(2.0 * qmul(mu_r, qconj(mu_d)) + C1 * one) / (qabs(mu_r) ** 2 + qabs(mu_d) ** 2 + C1)
    cs = qabs(2.0 * cor + C2 * one) / (var_r + var_d + C2)
    return float(lum), float(cs), float(lum * cs)


def qssim(tri_ref, tri_dis, K1: float = 0.01, K2: float = 0.03, L: float = 255.0) -> float:
    """QSSIM of one picture pair (see qssim_terms)."""
    return qssim_terms(tri_ref, tri_dis, K1, K2, L)[2]
