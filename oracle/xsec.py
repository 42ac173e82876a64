"""Velocity dependence of the cross section beyond the power law (oracle, FP64; test
infrastructure: only tests/ use it).

Sec. 2.4 fixes the method's two cross sections, the total sigma(v) for the Monte Carlo's
probability (Eq. dm-update-prob) and the momentum-transfer sigma_bar(v) for the gas's rates
(Eqs. scrA, scrB), and notes that any sigma(v) fits so long as A and B can be computed.  The
power law sigma0 (v / v0)^n has the closed forms of App. B; other laws go through the 1D
quadratures of oracle/rates.py (A_quad, B_quad, R_quad), which take any sigma_bar(u).

Families (params["xsec"], default "powerlaw"):
  * "powerlaw": sigma(v) = sigma0 (v / v0)^n (the closed forms are used);
  * "screened": sigma(v) = sigma0 / (1 + (v / v_c)^2)^2 with params["v_c_kms"], the velocity
    dependence of scattering through a massive mediator in the Born regime; it is flat below
    v_c and falls as v^-4 above it, so it reduces to the n = 0 power law for v_c -> infinity and
    to the n = -4 law sigma0 v_c^4 / v^4 for v >> v_c.
Both are isotropic unless params["beta"] != 0 (oracle/aniso.py), which scales sigma_bar by
1 - beta / 3.

Readings for the quadratures: w = 0 is evaluated at w = 1e-9 varsigma (A and B are even and
smooth in w, so the change is of relative order 1e-18); cold gas (varsigma = 0) takes the limits
A = sigma_bar(w) w, B = sigma_bar(w) w^3, R = sigma(w) w, as the closed forms do.

Parity: pinned by the reduction to the n = 0 closed forms (v_c -> infinity) and to the n = -4
law (v_c -> 0, scaled), the cold limits, sigma(v_c) = sigma0 / 4, and the Monte Carlo's mean
transfers against the quadrature expectations (tests/test_oracle_xsec.py).
"""
import numpy as np

from . import units
from .aniso import sbar_factor
from .rates import A_quad, B_quad, R_quad


def family(params):
    return params.get("xsec", "powerlaw")


def sigma_of_v(v, params):
    """Total cross section sigma(v) in kpc^2."""
    v = np.asarray(v, dtype=np.float64)
    s0 = units.sigma_kpc2(params["sigma0_cm2"])
    f = family(params)
    if f == "powerlaw":
        return s0 * (v / params["v0_kms"]) ** params["n"]
    if f == "screened":
        r = v / params["v_c_kms"]
        return s0 / (1.0 + r * r) ** 2
    raise ValueError(f"unknown cross-section family {f!r}")


def sigma_bar_of_v(v, params):
    """Momentum-transfer cross section sigma_bar(v) = sigma(v) (1 - beta / 3) in kpc^2."""
    return sigma_of_v(v, params) * sbar_factor(params.get("beta", 0.0))


def _rate_arr(fn, w, s2, sig, cold_power):
    w = np.asarray(w, dtype=np.float64)
    s2 = np.broadcast_to(np.asarray(s2, dtype=np.float64), w.shape)
    out = np.empty(w.shape)
    for k in range(w.size):
        wk, sk = float(w.flat[k]), float(s2.flat[k])
        if sk <= 0.0:
            out.flat[k] = float(sig(wk)) * wk ** cold_power
        else:
            out.flat[k] = fn(max(wk, 1e-9 * np.sqrt(sk)), sk, sig)
    return out


def A_arr(w, s2, params):
    """A(w; varsigma^2) of the family by quadrature, per element."""
    return _rate_arr(A_quad, w, s2, lambda u: float(sigma_bar_of_v(u, params)), 1)


def B_arr(w, s2, params):
    return _rate_arr(B_quad, w, s2, lambda u: float(sigma_bar_of_v(u, params)), 3)


def R_arr(w, s2, params):
    return _rate_arr(R_quad, w, s2, lambda u: float(sigma_of_v(u, params)), 1)
