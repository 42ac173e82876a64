"""One hierarchical substep with power-of-two timestep bins (oracle, FP64).

Test infrastructure: used only by tests/, the smoke check and the CPU baseline of bench.py.

Reading (the paper gives each DM particle a timestep limit through Eq. prob_criterion, Sec. 2.4,
and leaves the timestep hierarchy to the host code): a particle in bin b has dt = 2^b dt_min and
is active at substep s when s mod 2^b == 0.  At a substep
  * each active gas particle j receives the mean field (Eqs. gas-dVdt, gas-dTdt) of ALL its DM
    partners and is kicked with its own dt_j (u clamped at 0 as in oracle_step);
  * each active DM particle i draws the Monte Carlo (Eqs. dm-update-vels, dm-update-prob,
    scatter_chi) against ALL its gas partners with its own dt_i, Philox step = s;
  * every other particle is unchanged.
Both halves read the substep-start state (operator split, as in oracle_step).

Sums (as oracle_step, restricted to what moved): [0:3], [6], [9], [10], [13], [14] over the
active DM; [3:6], [7], [11] over the active gas; [8] the App. C expected DM energy change of
the pairs of the active gas over their dt_j; [12] half the pair evaluations
(pairs of active gas + pairs of active DM).

Parity: composed of pinned parts (meanfield.py, mc.py, expect.py); tests/test_oracle_step.py
checks that a substep with every particle in bin 0 is oracle_step.
"""
import numpy as np

from . import units
from .expect import expected_dm
from .kernel import overlap_g_vec
from .mc import mc_scatter
from .meanfield import meanfield_gas, pair_geometry
from .pairs import pairs_bruteforce


def active_mask(bins, substep):
    return (int(substep) % (2.0 ** bins.astype(np.float64))) == 0


def oracle_substep(dm, gas, params, substep, dt_min, dm_bin, gas_bin, pairs=None):
    if pairs is None:
        pairs = pairs_bruteforce(dm, gas, params["periodic"], params["box"])
    pi, pj = pairs
    act_d = active_mask(dm_bin, substep)
    act_g = active_mask(gas_bin, substep)
    dt_d = dt_min * 2.0 ** dm_bin.astype(np.float64)
    dt_g = dt_min * 2.0 ** gas_bin.astype(np.float64)
    d = pair_geometry(dm, gas, pi, pj, params["periodic"], params["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])

    # gas side: the mean field of the active gas rows
    mg = act_g[pj]
    acc, dudt = meanfield_gas(dm, gas, pi[mg], pj[mg], params, g[mg])
    acc[~act_g] = 0.0
    dudt[~act_g] = 0.0
    dtj = np.where(act_g, dt_g, 0.0)
    V_new = gas["vel"] + acc * dtj[:, None]
    u_old = units.u_from_T(gas["T"], gas["mu"])
    u_new = u_old + dudt * dtj
    u_clamped = act_g & (u_new < 0.0)
    u_new = np.where(u_clamped, 0.0, u_new)
    T_new = np.where(act_g, units.T_from_u(u_new, gas["mu"]), gas["T"])
    _, E_dE, _ = expected_dm(dm, gas, pi[mg], pj[mg], params, dt_g[pj[mg]], g[mg])

    # DM side: the Monte Carlo of the active DM rows, each with its own dt
    md = act_d[pi]
    mc = mc_scatter(dm, gas, pi[md], pj[md], params, substep, dt_d[pi[md]], g[md])

    Mi = dm["mass"]
    Mj = gas["mass"]
    v0 = dm["vel"]
    v1 = mc["vel_new"]
    sums = np.zeros(16)
    sums[0:3] = np.sum(Mi[:, None] * (v1 - v0), axis=0)
    sums[3:6] = np.sum(Mj[:, None] * acc * dtj[:, None], axis=0)
    sums[6] = np.sum(0.5 * Mi * (np.sum(v1 * v1, axis=1) - np.sum(v0 * v0, axis=1)))
    sums[7] = np.sum(Mj * (0.5 * (np.sum(V_new * V_new, axis=1) - np.sum(gas["vel"] ** 2, axis=1))
                           + u_new - u_old))
    sums[8] = np.sum(E_dE)
    sums[9] = np.count_nonzero(mc["scattered"])
    sums[10] = np.count_nonzero(mc["clamped"])
    sums[11] = np.count_nonzero(u_clamped)
    sums[12] = 0.5 * (np.count_nonzero(mg) + np.count_nonzero(md))
    sums[13] = np.sum(mc["P"])
    sums[14] = mc["p_ratio_max"].max() if len(Mi) else 0.0
    return dict(acc=acc, dudt=dudt, V_new=V_new, u_new=u_new, T_new=T_new, mc=mc, sums=sums,
                active_dm=act_d, active_gas=act_g, pairs=(pi, pj), g=g)


def rebin(ratio, bins, max_bin, substep=0, active=None):
    """New timestep bins from the criterion of Eq. prob_criterion (the dt feedback of Sec. 2.5:
    a particle whose P_ij is too large takes a smaller timestep next).

    ratio: float32 max_j P_ij / min(0.1, 1e-4 ((m_chi + mu_j) / mu_j)^2) of each particle at its
    current dt_i = 2^b dt_min (the Monte Carlo's p_ratio_max); P_ij is proportional to dt, so the
    ratio at bin b' is ratio 2^(b' - b).  Rule (the paper gives the criterion, not the bin
    arithmetic; this is the reading):
      * ratio > 1 (or not finite): the largest b' <= b with ratio 2^(b' - b) <= 1, at least 0:
        b' = b - k with k = ceil(log2 ratio), from ratio = m 2^e (m in [1/2, 1)): k = e, or
        e - 1 when m = 1/2 (ratio an exact power of two);
      * ratio < 1/4, b < max_bin and the next substep a multiple of 2^(b+1) (the larger step
        starts at a boundary of the hierarchy): b' = b + 1;
      * otherwise b' = b.  Inactive particles (active given and 0) keep their bins.
    """
    r = np.asarray(ratio, dtype=np.float32)
    b = np.asarray(bins, dtype=np.int64)
    out = b.copy()
    for i in range(len(r)):
        if active is not None and not active[i]:
            continue
        x = r[i]
        if not np.isfinite(x) or x > 1.0:
            if not np.isfinite(x):
                out[i] = 0
                continue
            m, e = np.frexp(x)
            k = int(e) - 1 if m == 0.5 else int(e)
            out[i] = max(0, int(b[i]) - k)
        elif x < 0.25 and b[i] < max_bin and substep % (1 << (int(b[i]) + 1)) == 0:
            out[i] = b[i] + 1
    return out.astype(np.uint8)
