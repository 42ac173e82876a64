"""One hybrid interaction step with kicks and FP64 conservation sums (oracle).

Order (Sec. 2.4, operator split at the step start):
  1. pair set {d_ij < h_i + h_j}
  2. gas mean field (Eqs. gas-dVdt, gas-dTdt) from the step-start state
  3. DM Monte Carlo (Eqs. dm-update-vels, dm-update-prob, scatter_chi) from the
     step-start state
  4. kicks: V_j += a_j dt; u_j += du_j/dt dt with u_j = (3/2) k_B T_j/mu_j, clamped
     at u_j >= 0 (reading: a negative thermal energy after a kick is clamped and
     counted); T_j from u_j
  5. sums (float64), in Msun, km/s:
       [0:3]  sum_i M_i (v_i' - v_i)             realised DM momentum change
       [3:6]  sum_j M_j a_j dt                     gas momentum change
       [6]    sum_i M_i (|v_i'|^2 - |v_i|^2) / 2   realised DM kinetic-energy change
       [7]    sum_j M_j [(|V_j'|^2 - |V_j|^2)/2 + u_j' - u_j]   gas energy change
       [8]    sum_i E[dE_i]                        expected DM energy change (App. C)
       [9]    number of scatters
       [10]   number of DM particles with sum_j P_ij > 1 (renormalised)
       [11]   number of gas particles whose u was clamped at 0
       [12]   number of pairs
       [13]   sum_ij P_ij                          expected number of scatters given the draws
       [14]   max_i p_ratio_max_i
       [15]   0 (reserved)
Parity: pinned through its parts; tests/test_oracle_step.py checks the sums'
identities.
"""
import numpy as np

from . import units
from .expect import expected_dm
from .kernel import overlap_g_vec
from .mc import mc_scatter
from .meanfield import meanfield_gas, pair_geometry
from .pairs import pairs_bruteforce


def oracle_step(dm, gas, params, step, dt, pairs=None):
    if pairs is None:
        pairs = pairs_bruteforce(dm, gas, params["periodic"], params["box"])
    pi, pj = pairs
    d = pair_geometry(dm, gas, pi, pj, params["periodic"], params["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    acc, dudt = meanfield_gas(dm, gas, pi, pj, params, g)
    mc = mc_scatter(dm, gas, pi, pj, params, step, dt, g)
    _, E_dE, _ = expected_dm(dm, gas, pi, pj, params, dt, g)

    V_new = gas["vel"] + acc * dt
    u_old = units.u_from_T(gas["T"], gas["mu"])
    u_new = u_old + dudt * dt
    u_clamped = u_new < 0.0
    u_new = np.where(u_clamped, 0.0, u_new)
    T_new = units.T_from_u(u_new, gas["mu"])

    Mi = dm["mass"]
    Mj = gas["mass"]
    v0 = dm["vel"]
    v1 = mc["vel_new"]
    sums = np.zeros(16)
    sums[0:3] = np.sum(Mi[:, None] * (v1 - v0), axis=0)
    sums[3:6] = np.sum(Mj[:, None] * acc * dt, axis=0)
    sums[6] = np.sum(0.5 * Mi * (np.sum(v1 * v1, axis=1) - np.sum(v0 * v0, axis=1)))
    sums[7] = np.sum(Mj * (0.5 * (np.sum(V_new * V_new, axis=1) - np.sum(gas["vel"] ** 2, axis=1))
                           + u_new - u_old))
    sums[8] = np.sum(E_dE)
    sums[9] = np.count_nonzero(mc["scattered"])
    sums[10] = np.count_nonzero(mc["clamped"])
    sums[11] = np.count_nonzero(u_clamped)
    sums[12] = len(pi)
    sums[13] = np.sum(mc["P"])
    sums[14] = mc["p_ratio_max"].max() if len(Mi) else 0.0
    return dict(acc=acc, dudt=dudt, V_new=V_new, u_new=u_new, T_new=T_new, mc=mc, sums=sums,
                pairs=(pi, pj), g=g)
