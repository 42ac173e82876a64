"""Momentum- and energy-transfer integrals A, B and the total rate R (oracle, FP64).

Definitions (Eqs. scrA, scrB, with G the isotropic 3D Gaussian of variance varsigma^2):
    A(w; s2) = int d^3u G(w - u, s2) u (u.w / w^2) sigma_bar(u)
    B(w; s2) = int d^3u G(w - u, s2) u^3 sigma_bar(u)
and the Maxwellian-averaged total rate that the Monte Carlo probability averages to
(Eq. dm-update-prob averaged over v_B):
    R(w; s2) = int d^3u G(w - u, s2) u sigma(u).

Closed forms (App. B) for sigma_bar(v) = sigma0 (v / v0)^n, integer n >= -4:
    A = (alpha_n / 3) (sigma0 / v0^n) s^(n+1) 1F1(-(n+1)/2, 5/2; -x)
    B =  alpha_n      (sigma0 / v0^n) s^(n+3) 1F1(-(n+3)/2, 3/2; -x)
    alpha_n = 2^((n+5)/2) Gamma(3 + n/2) / sqrt(pi),   x = w^2 / (2 s^2),  s = varsigma.
R follows from the Gaussian moment <u^m> = s^m 2^(m/2) Gamma((m+3)/2)/Gamma(3/2)
1F1(-m/2, 3/2; -x) with m = n + 1 (diverges for n = -4).

Readings: w = 0 uses x = 0 (1F1 = 1); cold gas (varsigma = 0) uses the limits
A = sigma_bar(w) w, B = sigma_bar(w) w^3, R = sigma(w) w.

The 1D quadrature (any sigma_bar) integrates the angle analytically, with
C = 4 pi (2 pi s^2)^(-3/2) and k = u w / s^2:
    A = C int_0^inf du u^4 sigma_bar(u) / w  e^(-(u^2+w^2)/2s^2) i1(k),   i1(k) = cosh k / k - sinh k / k^2
    B = C int_0^inf du u^5 sigma_bar(u)      e^(-(u^2+w^2)/2s^2) sinh k / k
    R = C int_0^inf du u^3 sigma(u)          e^(-(u^2+w^2)/2s^2) sinh k / k
evaluated by adaptive Gauss-Kronrod (scipy.integrate.quad) with the exponentials
scaled so nothing overflows.

Parity: pinned.  tests/test_oracle_rates.py checks closed form == quadrature,
the w -> 0 values, the cold limits, n = 0 R against its erf form
s sqrt(2/pi) e^-x + (w + s^2/w) erf(w / (sqrt 2 s)), and a Monte Carlo estimate
of the 3D definitions.
"""
import math

import numpy as np
from scipy import integrate

from .hyp1f1 import hyp1f1_neg


def alpha_n(n):
    """alpha_n = 2^((n+5)/2) Gamma(3 + n/2) / sqrt(pi)  (App. B)."""
    return 2.0 ** ((n + 5) / 2.0) * math.gamma(3.0 + n / 2.0) / math.sqrt(math.pi)


def sigma_powerlaw(v, sigma0, v0, n):
    """sigma(v) = sigma0 (v / v0)^n (Sec. 2.4, isotropic so sigma = sigma_bar)."""
    return sigma0 * (np.asarray(v, dtype=np.float64) / v0) ** n


def A_closed(w, s2, sigma0, v0, n):
    """A(w; varsigma^2) from the App. B closed form, scalar inputs."""
    w = float(w)
    s2 = float(s2)
    if s2 == 0.0:
        return float(sigma_powerlaw(w, sigma0, v0, n)) * w
    s = math.sqrt(s2)
    x = w * w / (2.0 * s2)
    return alpha_n(n) / 3.0 * sigma0 / v0 ** n * s ** (n + 1) * hyp1f1_neg(-(n + 1) / 2.0, 2.5, x)


def B_closed(w, s2, sigma0, v0, n):
    """B(w; varsigma^2) from the App. B closed form, scalar inputs."""
    w = float(w)
    s2 = float(s2)
    if s2 == 0.0:
        return float(sigma_powerlaw(w, sigma0, v0, n)) * w ** 3
    s = math.sqrt(s2)
    x = w * w / (2.0 * s2)
    return alpha_n(n) * sigma0 / v0 ** n * s ** (n + 3) * hyp1f1_neg(-(n + 3) / 2.0, 1.5, x)


def R_closed(w, s2, sigma0, v0, n):
    """Maxwellian-averaged <sigma(u) u> for the power law (n > -4)."""
    if n <= -4:
        raise ValueError("the averaged total rate diverges for n <= -4")
    w = float(w)
    s2 = float(s2)
    if s2 == 0.0:
        return float(sigma_powerlaw(w, sigma0, v0, n)) * w
    s = math.sqrt(s2)
    x = w * w / (2.0 * s2)
    m = n + 1
    pref = 2.0 ** (m / 2.0) * math.gamma((m + 3) / 2.0) / math.gamma(1.5)
    return sigma0 / v0 ** n * s ** m * pref * hyp1f1_neg(-m / 2.0, 1.5, x)


def _vec(fn, w, s2, *args):
    w = np.asarray(w, dtype=np.float64)
    s2 = np.broadcast_to(np.asarray(s2, dtype=np.float64), w.shape)
    out = np.empty(w.shape)
    fo, fw, fs = out.reshape(-1), w.reshape(-1), s2.reshape(-1)
    for k in range(fw.size):
        fo[k] = fn(fw[k], fs[k], *args)
    return out


def A_closed_vec(w, s2, sigma0, v0, n):
    return _vec(A_closed, w, s2, sigma0, v0, n)


def B_closed_vec(w, s2, sigma0, v0, n):
    return _vec(B_closed, w, s2, sigma0, v0, n)


def R_closed_vec(w, s2, sigma0, v0, n):
    return _vec(R_closed, w, s2, sigma0, v0, n)


# ---- 1D quadrature ------------------------------------------------------------

def _angular_kernels(u, w, s2):
    """Return (e^-(u^2+w^2)/2s2 sinh k / k, e^-(u^2+w^2)/2s2 i1(k)) without overflow."""
    k = u * w / s2
    em = math.exp(-(u - w) ** 2 / (2.0 * s2))  # e^-(u^2+w^2)/2s2 * e^{+k}
    ep = math.exp(-(u + w) ** 2 / (2.0 * s2))  # e^-(u^2+w^2)/2s2 * e^{-k}
    if k < 0.5:
        # Taylor series: sinh k / k = sum k^2m / (2m+1)!,  i1(k) = sum 2m k^(2m-1) / (2m+1)!
        base = math.exp(-(u * u + w * w) / (2.0 * s2))
        sinhk_k = 0.0
        i1 = 0.0
        for m in range(12):
            f = math.factorial(2 * m + 1)
            sinhk_k += k ** (2 * m) / f
            if m > 0:
                i1 += 2.0 * m * k ** (2 * m - 1) / f
        return base * sinhk_k, base * i1
    sinhk_k = (em - ep) / (2.0 * k)
    i1 = 0.5 * (em * (1.0 / k - 1.0 / (k * k)) + ep * (1.0 / k + 1.0 / (k * k)))
    return sinhk_k, i1


def _quad(f, w, s2):
    s = math.sqrt(s2)
    lo = max(0.0, w - 40.0 * s)
    hi = w + 40.0 * s
    pts = [p for p in (w, w - 5 * s, w + 5 * s) if lo < p < hi]
    val, _ = integrate.quad(f, lo, hi, points=pts or None, epsabs=0.0, epsrel=1e-13, limit=400)
    if lo > 0.0:
        return val
    return val


def A_quad(w, s2, sigma_bar):
    """A by 1D quadrature for any sigma_bar(u) callable (w > 0, s2 > 0)."""
    C = 4.0 * math.pi * (2.0 * math.pi * s2) ** -1.5
    return C * _quad(lambda u: u ** 4 * sigma_bar(u) / w * _angular_kernels(u, w, s2)[1], w, s2)


def B_quad(w, s2, sigma_bar):
    """B by 1D quadrature."""
    C = 4.0 * math.pi * (2.0 * math.pi * s2) ** -1.5
    return C * _quad(lambda u: u ** 5 * sigma_bar(u) * _angular_kernels(u, w, s2)[0], w, s2)


def R_quad(w, s2, sigma):
    """R = <sigma(u) u> by 1D quadrature."""
    C = 4.0 * math.pi * (2.0 * math.pi * s2) ** -1.5
    return C * _quad(lambda u: u ** 3 * sigma(u) * _angular_kernels(u, w, s2)[0], w, s2)


def _closed_arr(w, s2, sigma0, v0, n, which):
    from .hyp1f1 import hyp1f1_neg_arr
    w = np.asarray(w, dtype=np.float64)
    s2 = np.broadcast_to(np.asarray(s2, dtype=np.float64), w.shape)
    out = np.empty(w.shape)
    cold = s2 == 0.0
    hot = ~cold
    s = np.sqrt(s2[hot])
    x = w[hot] ** 2 / (2.0 * s2[hot])
    if which == "A":
        out[hot] = alpha_n(n) / 3.0 * sigma0 / v0 ** n * s ** (n + 1) * hyp1f1_neg_arr(-(n + 1) / 2.0, 2.5, x)
        out[cold] = sigma_powerlaw(w[cold], sigma0, v0, n) * w[cold]
    elif which == "B":
        out[hot] = alpha_n(n) * sigma0 / v0 ** n * s ** (n + 3) * hyp1f1_neg_arr(-(n + 3) / 2.0, 1.5, x)
        out[cold] = sigma_powerlaw(w[cold], sigma0, v0, n) * w[cold] ** 3
    else:
        if n <= -4:
            raise ValueError("the averaged total rate diverges for n <= -4")
        m = n + 1
        pref = 2.0 ** (m / 2.0) * math.gamma((m + 3) / 2.0) / math.gamma(1.5)
        out[hot] = sigma0 / v0 ** n * s ** m * pref * hyp1f1_neg_arr(-m / 2.0, 1.5, x)
        out[cold] = sigma_powerlaw(w[cold], sigma0, v0, n) * w[cold]
    return out


def A_closed_arr(w, s2, sigma0, v0, n):
    """Array version of A_closed (same formula, vectorised 1F1)."""
    return _closed_arr(w, s2, sigma0, v0, n, "A")


def B_closed_arr(w, s2, sigma0, v0, n):
    """Array version of B_closed."""
    return _closed_arr(w, s2, sigma0, v0, n, "B")


def R_closed_arr(w, s2, sigma0, v0, n):
    """Array version of R_closed."""
    return _closed_arr(w, s2, sigma0, v0, n, "R")
