"""Pins for the oracle's cubic-spline kernel and overlap integral (Sec. 2.4, App. D)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernel as K


def test_kernel_integrates_to_one():
    # Sec. 2.4: the cubic spline integrates to 1 (closed form: 4 pi int r^2 W dr)
    for h in (0.3, 1.0, 7.5):
        v, _ = integrate.quad(lambda r: 4 * math.pi * r * r * K.W(np.array([r]), h)[0], 0, h,
                              points=[h / 2], epsabs=0, epsrel=1e-13)
        assert abs(v - 1.0) < 1e-12


def test_kernel_piecewise_values():
    # values straight from the printed piecewise form at q = 0, 1/4, 1/2, 3/4, 1, 1.2
    h = 2.0
    q = np.array([0.0, 0.25, 0.5, 0.75, 1.0, 1.2])
    expect = 8 / (math.pi * h ** 3) * np.array([1.0, 1 - 6 / 16 + 6 / 64, 1 - 6 / 4 + 6 / 8,
                                                2 * 0.25 ** 3, 0.0, 0.0])
    np.testing.assert_allclose(K.W(q * h, h), expect, rtol=1e-15, atol=0)


@pytest.mark.parametrize("hi,hj", [(1.0, 1.0), (1.0, 0.6), (0.3, 1.0), (1.0, 0.05)])
def test_overlap_normalised(hi, hj):
    # g is the convolution of two unit-normalised kernels: int g(d) d^3 d = 1
    f = lambda d: 4 * math.pi * d * d * K.overlap_g(d, hi, hj)
    a, b = max(hi, hj), min(hi, hj)
    pts = sorted({abs(a - b), a, b, 0.5 * a, a - 0.5 * b, a + 0.5 * b, a - b / 2})
    pts = [p for p in pts if 0 < p < a + b]
    v, _ = integrate.quad(f, 0, a + b, points=pts, epsabs=0, epsrel=1e-12, limit=500)
    assert abs(v - 1.0) < 1e-10


def _g_direct(d, h_center, h_other):
    """Unsubstituted App. D form: 2 pi int r^2 W(r, h_center) int dc W(|x - d z|, h_other),
    integrated numerically in (r, c) with no analytic step."""
    def inner(r):
        f = lambda c: K.W(np.array([math.sqrt(max(r * r + d * d - 2 * d * r * c, 0.0))]), h_other)[0]
        # the integrand has kinks where |x - d z| = h_other/2 and h_other
        kinks = []
        if d > 0 and r > 0:
            for rho in (0.5 * h_other, h_other):
                c = (r * r + d * d - rho * rho) / (2 * d * r)
                if -1 < c < 1:
                    kinks.append(c)
        v, _ = integrate.quad(f, -1, 1, points=kinks or None, epsabs=1e-14, epsrel=1e-11, limit=200)
        return r * r * K.W(np.array([r]), h_center)[0] * v
    kinks = [p for p in (0.5 * h_center, abs(d - h_other), abs(d - h_other / 2), d,
                         d + h_other / 2) if 0 < p < h_center]
    v, _ = integrate.quad(inner, 0, h_center, points=kinks or None, epsabs=1e-14, epsrel=1e-10, limit=200)
    return 2 * math.pi * v


@pytest.mark.parametrize("d,hi,hj", [(0.0, 1.0, 0.7), (0.001, 1.0, 0.7), (0.35, 1.0, 0.7),
                                     (1.2, 1.0, 0.7), (0.9, 0.5, 1.0), (0.2, 1.0, 0.1)])
def test_overlap_matches_direct_2d_quadrature(d, hi, hj):
    ref_ij = _g_direct(d, hi, hj)   # kernel i at the origin
    ref_ji = _g_direct(d, hj, hi)   # roles swapped: checks symmetry and the h ordering
    g = K.overlap_g(d, hi, hj)
    assert abs(ref_ij - ref_ji) < 1e-8 * abs(ref_ij)
    assert abs(g - ref_ij) < 1e-8 * abs(ref_ij)


def test_overlap_small_partner_limit():
    # h_j / h_i -> 0: the partner kernel becomes a delta function, g -> W(d, h_i)
    # and the leading correction is second order in h_j (smoothing by a narrow kernel)
    hi = 1.0
    for d in (0.1, 0.4, 0.6, 0.9):
        w = K.W(np.array([d]), hi)[0]
        e3 = K.overlap_g(d, hi, 1e-3) / w - 1.0
        e4 = K.overlap_g(d, hi, 1e-4) / w - 1.0
        assert abs(e4) < 1e-6
        assert 80.0 < e3 / e4 < 120.0


def test_overlap_support_and_positivity():
    assert K.overlap_g(1.7, 1.0, 0.7) == 0.0
    assert K.overlap_g(1.7000001, 1.0, 0.7) == 0.0
    assert K.overlap_g(1.6999, 1.0, 0.7) > 0.0
    assert K.overlap_g(0.0, 1.0, 1.0) > K.overlap_g(0.5, 1.0, 1.0) > K.overlap_g(1.5, 1.0, 1.0) > 0


def test_overlap_scaling():
    # g has dimensions of inverse volume: g(l d; l h_i, l h_j) = g(d; h_i, h_j) / l^3
    for l in (0.01, 3.0):
        assert abs(K.overlap_g(0.3 * l, 1.0 * l, 0.5 * l) * l ** 3 - K.overlap_g(0.3, 1.0, 0.5)) < 1e-13


def test_overlap_equal_kernels_at_zero_separation():
    # g(0; h, h) = int W^2 d^3x, computed here by 1D quadrature of the kernel alone
    h = 1.3
    v, _ = integrate.quad(lambda r: 4 * math.pi * r * r * K.W(np.array([r]), h)[0] ** 2, 0, h,
                          points=[h / 2], epsabs=0, epsrel=1e-13)
    assert abs(K.overlap_g(0.0, h, h) - v) < 1e-12 * v


def test_overlap_vectorised_equals_scalar():
    rng = np.random.default_rng(5)
    hi = rng.uniform(0.02, 1.0, 400)
    hj = rng.uniform(0.02, 1.0, 400)
    d = rng.uniform(0, 1.05, 400) * (hi + hj)
    d[:5] = 0.0
    np.testing.assert_allclose(K.overlap_g_vec(d, hi, hj), K.overlap_g_many(d, hi, hj),
                               rtol=1e-13, atol=0)


def test_planted_kernel_mistake_is_caught(monkeypatch):
    # a plausible slip (outer piece 2(1-q)^2 instead of 2(1-q)^3) must break the normalisation pin
    orig = K.w_unit

    def wrong(u):
        u = np.asarray(u, dtype=np.float64)
        out = orig(u)
        outer = (u > 0.5) & (u <= 1.0)
        out[outer] = 8 / np.pi * 2 * (1 - u[outer]) ** 2
        return out

    monkeypatch.setattr(K, "w_unit", wrong)
    f = lambda d: 4 * math.pi * d * d * K.overlap_g(d, 1.0, 0.6)
    v, _ = integrate.quad(f, 0, 1.6, limit=200, points=[0.3, 0.4, 0.5, 0.7, 1.0, 1.3])
    assert abs(v - 1.0) > 1e-3
