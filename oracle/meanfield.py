"""Gas mean-field momentum and energy transfer (oracle, FP64).

Eq. gas-dVdt:  dV_j/dt = sum_i M_i/(m_chi + mu_j) g_ij A(w_ij; T_j/mu_j) w_ij
Eq. gas-dTdt:  (3/(2 mu_j)) dT_j/dt
             = sum_i M_i/(m_chi + mu_j) g_ij [ w_ij^2 A - mu_j/(m_chi + mu_j) B ]
with w_ij = v_i - V_j.  In code units the left side of the second equation is
du_j/dt, u_j = (3/2) k_B T_j / mu_j the specific thermal energy.  Sums run over
each gas particle's DM partners in ascending DM index.

Both sides read the state at the start of the step (operator split).

Parity: pinned through its parts (kernel.py, rates.py) and through the App. C
identities checked in tests/test_oracle_step.py.
"""
import numpy as np

from . import units
from .aniso import sbar_factor
from .kernel import overlap_g_vec
from .pairs import min_image
from .rates import A_closed_arr, B_closed_arr
from .xsec import A_arr, B_arr, family


def pair_geometry(dm, gas, pi, pj, periodic, box):
    dx = dm["pos"][pi] - gas["pos"][pj]
    if periodic:
        dx = min_image(dx, box)
    d = np.sqrt(np.sum(dx * dx, axis=1))
    return d


def pair_rates(dm, gas, pi, pj, params, g=None):
    """Per-pair (g, w vector, A, B) in code units; A, B carry sigma in kpc^2."""
    if g is None:
        d = pair_geometry(dm, gas, pi, pj, params["periodic"], params["box"])
        g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    w = dm["vel"][pi] - gas["vel"][pj]
    wn = np.sqrt(np.sum(w * w, axis=1))
    s2 = units.varsigma2_kms2(gas["T"][pj], gas["mu"][pj])
    if family(params) != "powerlaw":                # other sigma(v): quadrature (oracle/xsec.py)
        return g, w, A_arr(wn, s2, params), B_arr(wn, s2, params)
    # the exchange rates take the momentum-transfer cross section (oracle/aniso.py)
    sig0 = units.sigma_kpc2(params["sigma0_cm2"]) * sbar_factor(params.get("beta", 0.0))
    A = A_closed_arr(wn, s2, sig0, params["v0_kms"], params["n"])
    B = B_closed_arr(wn, s2, sig0, params["v0_kms"], params["n"])
    return g, w, A, B


def meanfield_gas(dm, gas, pi, pj, params, g=None):
    """Return (acc[N_B, 3], dudt[N_B]) in code units ((km/s)^2/kpc and (km/s)^3/kpc)."""
    m_chi = params["m_chi_mp"]
    g, w, A, B = pair_rates(dm, gas, pi, pj, params, g)
    mu = gas["mu"][pj]
    # M_i / (m_chi + mu_j): Msun -> number of particles of mass (m_chi + mu_j) m_p
    coef = dm["mass"][pi] * units.MSUN_PER_MP / (m_chi + mu) * g
    w2 = np.sum(w * w, axis=1)
    acc_terms = (coef * A)[:, None] * w
    dudt_terms = coef * (w2 * A - mu / (m_chi + mu) * B)
    nb = len(gas["h"])
    order = np.lexsort((pi, pj))          # per gas, ascending DM index
    acc = np.zeros((nb, 3))
    dudt = np.zeros(nb)
    # ufunc.at applies the additions one by one in the given order: plain
    # sequential FP64 sums per gas particle, ascending DM index.
    for c in range(3):
        np.add.at(acc[:, c], pj[order], acc_terms[order, c])
    np.add.at(dudt, pj[order], dudt_terms[order])
    return acc, dudt
