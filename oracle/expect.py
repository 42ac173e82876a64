"""Expected DM transfers and the pairwise conservation identities (App. C, oracle).

App. C:  E[dv_i] = sum_j M_j/(m_chi + mu_j) g_ij A(w_ij) (V_j - v_i) dt
         E[dE_i] = M_i sum_j M_j/(m_chi + mu_j) g_ij [ mu_j/(m_chi + mu_j) B(w_ij)
                                                       - v_i.(v_i - V_j) A(w_ij) ] dt
and for every pair (i, j):
         M_i E[dv_i] + M_j dV_j/dt dt = 0
         E[dE_i] + (3 M_j / (2 mu_j)) dT_j/dt dt + M_j V_j . dV_j/dt dt = 0.
The expected scatter probability of DM i is sum_j (M_j/mu_j) g_ij R(w_ij) dt, the
Maxwellian average of P_ij (Eq. dm-update-prob averaged over v^B).

Parity: pinned by the identities themselves (tests/test_oracle_step.py) and by
the statistical test of the MC against these expectations.
"""
import numpy as np

from . import units
from .meanfield import pair_rates
from .rates import R_closed_arr
from .xsec import R_arr, family


def expected_dm(dm, gas, pi, pj, params, dt, g=None):
    """Return (E_dv[N_chi,3], E_dE[N_chi], E_P[N_chi]) (E_P needs n > -4, else NaN)."""
    m_chi = params["m_chi_mp"]
    g, w, A, B = pair_rates(dm, gas, pi, pj, params, g)
    mu = gas["mu"][pj]
    coef = gas["mass"][pj] * units.MSUN_PER_MP / (m_chi + mu) * g * dt
    vi = dm["vel"][pi]
    dv_terms = (coef * A)[:, None] * (-w)
    dE_terms = dm["mass"][pi] * coef * (mu / (m_chi + mu) * B - np.sum(vi * w, axis=1) * A)
    nd = len(dm["h"])
    E_dv = np.zeros((nd, 3))
    E_dE = np.zeros(nd)
    order = np.lexsort((gas["id"][pj], pi))
    for c in range(3):
        np.add.at(E_dv[:, c], pi[order], dv_terms[order, c])
    np.add.at(E_dE, pi[order], dE_terms[order])
    E_P = np.full(nd, np.nan)
    if family(params) != "powerlaw" or params["n"] > -4:
        s2 = units.varsigma2_kms2(gas["T"][pj], gas["mu"][pj])
        wn = np.sqrt(np.sum(w * w, axis=1))
        if family(params) != "powerlaw":
            R = R_arr(wn, s2, params)
        else:
            R = R_closed_arr(wn, s2, units.sigma_kpc2(params["sigma0_cm2"]), params["v0_kms"], params["n"])
        nB = gas["mass"][pj] * units.MSUN_PER_MP / mu
        E_P = np.zeros(nd)
        np.add.at(E_P, pi[order], (nB * g * R * dt)[order])
    return E_dv, E_dE, E_P


def pair_budget(dm, gas, pi, pj, params, dt, g=None):
    """Per-pair momentum and energy residuals of the App. C identities.

    Returns (dp[npairs,3], dE[npairs], scale_p[npairs], scale_E[npairs]) where
    dp = M_i E[dv_i]_ij + M_j (dV_j/dt)_ij dt and dE likewise; the scales are the
    magnitudes of the individual terms, for relative comparisons.
    """
    m_chi = params["m_chi_mp"]
    g, w, A, B = pair_rates(dm, gas, pi, pj, params, g)
    mu = gas["mu"][pj]
    Mi = dm["mass"][pi]
    Mj = gas["mass"][pj]
    # DM side (App. C)
    dv_i = (Mj * units.MSUN_PER_MP / (m_chi + mu) * g * A * dt)[:, None] * (-w)
    dE_i = Mi * Mj * units.MSUN_PER_MP / (m_chi + mu) * g * dt * (
        mu / (m_chi + mu) * B - np.sum(dm["vel"][pi] * w, axis=1) * A)
    # gas side (Eqs. gas-dVdt, gas-dTdt)
    coef = Mi * units.MSUN_PER_MP / (m_chi + mu) * g
    a_j = (coef * A)[:, None] * w
    dudt_j = coef * (np.sum(w * w, axis=1) * A - mu / (m_chi + mu) * B)
    Vj = gas["vel"][pj]
    dp = Mi[:, None] * dv_i + Mj[:, None] * a_j * dt
    dE = dE_i + Mj * dudt_j * dt + Mj * np.sum(Vj * a_j, axis=1) * dt
    scale_p = np.abs(Mi[:, None] * dv_i).max(axis=1)
    scale_E = np.abs(dE_i) + np.abs(Mj * dudt_j * dt) + np.abs(Mj * np.sum(Vj * a_j, axis=1) * dt)
    return dp, dE, scale_p, scale_E
