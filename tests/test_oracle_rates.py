"""Pins for the oracle's 1F1, A, B and R (Sec. 2.4, Eqs. scrA/scrB, App. B)."""
import math
import warnings

import numpy as np
import pytest
from scipy import special

from oracle import hyp1f1 as H
from oracle import rates as Rt

mpmath = pytest.importorskip("mpmath")

XS = [0.0, 1e-9, 1e-4, 0.03, 0.7, 3.0, 12.0, 33.0, 49.99, 50.0, 50.01, 77.0, 300.0, 2500.0, 1e4]


def _cases():
    out = []
    for n in range(-4, 5):
        for a, b in ((-(n + 1) / 2, 2.5), (-(n + 3) / 2, 1.5), (-(n + 1) / 2, 1.5)):
            if b - a > 0:
                out.append((n, a, b))
    return out


@pytest.mark.parametrize("n,a,b", _cases())
def test_hyp1f1_against_mpmath(n, a, b):
    mpmath.mp.dps = 40
    for x in XS:
        ref = float(mpmath.hyp1f1(a, b, -x))
        v = H.hyp1f1_neg(a, b, x)
        assert abs(v - ref) <= 2e-14 * abs(ref), (x, v, ref)


def test_hyp1f1_erf_special_case():
    # 1F1(1/2, 3/2; -x) = (sqrt(pi)/2) erf(sqrt x)/sqrt x  (DLMF 13.6.7 / 7.11.4)
    for x in [1e-6, 0.01, 1.0, 10.0, 49.0, 51.0, 400.0]:
        ref = math.sqrt(math.pi) / 2 * math.erf(math.sqrt(x)) / math.sqrt(x)
        assert abs(H.hyp1f1_neg(0.5, 1.5, x) - ref) < 1e-14 * ref


def test_hyp1f1_seam_is_continuous():
    for n, a, b in _cases():
        # both branches evaluated at the switch point agree (the series is positive,
        # the large-x form drops only the e^-x part, ~1e-22 relative here)
        lo = H._kummer_series(a, b, 50.0)
        hi = H._asymptotic(a, b, 50.0)
        assert abs(lo - hi) < 1e-13 * abs(hi)


def test_hyp1f1_array_equals_scalar():
    rng = np.random.default_rng(2)
    x = np.concatenate([10 ** rng.uniform(-6, 4, 3000), [0.0, 50.0]])
    for n, a, b in _cases():
        np.testing.assert_allclose(H.hyp1f1_neg_arr(a, b, x), H.hyp1f1_neg_vec(a, b, x), rtol=1e-14)


@pytest.mark.parametrize("n", [-4, -3, -2, -1, 0, 1, 2, 3])
def test_closed_forms_match_quadrature(n):
    sb = lambda u: (u / 100.0) ** n
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for w in (0.01, 0.5, 9.0, 30.0, 100.0, 300.0, 2000.0):
            for s2 in (81.0, 1e4):
                assert abs(Rt.A_closed(w, s2, 1.0, 100.0, n) / Rt.A_quad(w, s2, sb) - 1) < 1e-12
                assert abs(Rt.B_closed(w, s2, 1.0, 100.0, n) / Rt.B_quad(w, s2, sb) - 1) < 1e-12
                if n > -4:
                    assert abs(Rt.R_closed(w, s2, 1.0, 100.0, n) / Rt.R_quad(w, s2, sb) - 1) < 1e-12


@pytest.mark.parametrize("n", [-4, -2, 0, 2])
def test_rest_values(n):
    # w = 0: 1F1 = 1, so A = (alpha_n/3) s^(n+1), B = alpha_n s^(n+3) (sigma0 = v0 = 1);
    # and directly <u^m> of a centred Maxwellian = s^m 2^(m/2) Gamma((m+3)/2)/Gamma(3/2)
    s2 = 2.3
    s = math.sqrt(s2)
    mom = lambda m: s ** m * 2 ** (m / 2) * math.gamma((m + 3) / 2) / math.gamma(1.5)
    assert abs(Rt.B_closed(0.0, s2, 1.0, 1.0, n) - mom(n + 3)) < 1e-13 * mom(n + 3)
    # A(w) w = <u^(n+1) u_z> along w = w z; its slope at w = 0 is, by differentiating the
    # Gaussian, <u^(n+1) u_z^2>_0 / s^2 = <u^(n+3)>_0 / (3 s^2), so A(0) = <u^(n+3)>/(3 s^2)
    a0 = mom(n + 3) / (3 * s2)
    assert abs(Rt.A_closed(0.0, s2, 1.0, 1.0, n) - a0) < 1e-13 * a0


@pytest.mark.parametrize("n", [-4, -2, 0, 2])
def test_cold_limits(n):
    # varsigma -> 0: A -> sigma(w) w and B -> sigma(w) w^3 (all gas at V_j)
    w = 150.0
    sig = (w / 100.0) ** n
    for s2 in (1e-2, 1e-4):
        a = Rt.A_closed(w, s2, 1.0, 100.0, n)
        b = Rt.B_closed(w, s2, 1.0, 100.0, n)
        rel = 10 * s2 / w ** 2 * (abs(n) + 3) ** 2
        assert abs(a / (sig * w) - 1) < rel
        assert abs(b / (sig * w ** 3) - 1) < rel
    assert Rt.A_closed(w, 0.0, 1.0, 100.0, n) == sig * w


def test_R_n0_erf_form():
    # <u> for a Maxwellian offset by w: s sqrt(2/pi) e^-x + (w + s^2/w) erf(w/(sqrt2 s))
    for w, s2 in ((0.3, 4.0), (9.0, 81.0), (200.0, 81.0), (1.0, 1e4)):
        s = math.sqrt(s2)
        x = w * w / (2 * s2)
        ref = s * math.sqrt(2 / math.pi) * math.exp(-x) + (w + s2 / w) * math.erf(w / (math.sqrt(2) * s))
        assert abs(Rt.R_closed(w, s2, 1.0, 1.0, 0) - ref) < 1e-13 * ref


@pytest.mark.parametrize("n", [-2, 0, 2])
def test_monte_carlo_of_3d_definitions(n):
    # brute-force sampling of Eqs. scrA/scrB: u = w + s z, z ~ N(0, I)
    rng = np.random.default_rng(11 + n)
    wv = np.array([30.0, -12.0, 5.0])
    wn = np.linalg.norm(wv)
    s2 = 400.0
    N = 2_000_000
    u = wv[None, :] + math.sqrt(s2) * rng.standard_normal((N, 3))
    un = np.linalg.norm(u, axis=1)
    sb = (un / 100.0) ** n
    fa = un * (u @ wv) / wn ** 2 * sb
    fb = un ** 3 * sb
    fr = un * sb
    for f, ref in ((fa, Rt.A_closed(wn, s2, 1.0, 100.0, n)), (fb, Rt.B_closed(wn, s2, 1.0, 100.0, n)),
                   (fr, Rt.R_closed(wn, s2, 1.0, 100.0, n))):
        est = f.mean()
        err = f.std() / math.sqrt(N)
        assert abs(est - ref) < 5 * err, (est, ref, err)


def test_alpha_n_values():
    # alpha_0 = 2^(5/2) Gamma(3)/sqrt(pi) = 8 sqrt(2/pi)
    assert abs(Rt.alpha_n(0) - 8 * math.sqrt(2 / math.pi)) < 1e-15
    assert abs(Rt.alpha_n(-4) - math.sqrt(2 / math.pi)) < 1e-15


def test_array_forms_equal_scalar():
    rng = np.random.default_rng(4)
    w = 10 ** rng.uniform(-2, 3.5, 500)
    s2 = 10 ** rng.uniform(0, 4, 500)
    s2[:3] = 0.0
    for n in (-4, -2, 0, 2):
        np.testing.assert_allclose(Rt.A_closed_arr(w, s2, 1.0, 100.0, n),
                                   Rt.A_closed_vec(w, s2, 1.0, 100.0, n), rtol=1e-14)
        np.testing.assert_allclose(Rt.B_closed_arr(w, s2, 1.0, 100.0, n),
                                   Rt.B_closed_vec(w, s2, 1.0, 100.0, n), rtol=1e-14)
