"""DM Monte Carlo scattering (oracle, FP64).

Eq. dm-update-vels: the new velocity distribution of DM particle i is
    nu_i' = (1 - sum_j P_ij) delta(v - v_i) + sum_j P_ij delta(v - S_chi(v_i, v^B_ij, Omega_ij))
Eq. dm-update-prob:  P_ij = (M_j / mu_j) g_ij sigma(v_rel) v_rel dt,  v_rel = |v_i - v^B_ij|
with v^B_ij one sample of the gas Maxwellian G(v - V_j, T_j/mu_j) per pair, and
Eq. scatter_chi:     S_chi = v_i + mu_j/(m_chi + mu_j) v_rel (n' - n),  n = (v_i - v^B)/v_rel,
n' isotropic (Sec. 2.4: isotropic power-law cross section), or, with params["beta"] != 0,
drawn from dsigma/dOmega proportional to 1 + beta cos theta about n (oracle/aniso.py); P_ij
keeps the total cross section sigma.

Readings (the paper leaves these open):
  * one categorical draw per DM particle per step (the derivation's form); partners
    in ascending gas id; running sums C_k = sum_{j<=k} P_ij; with r_i the DM
    stream's uniform the particle scatters off the first k with r_i < C_k.
  * if C_last > 1 the categorical is renormalised by C_last (the particle scatters
    surely, threshold r_i C_last) and the event is counted as a clamp.
  * Eq. prob_criterion: the output p_ratio_max_i = max_j P_ij / min(0.1,
    1e-4 ((m_chi + mu_j)/mu_j)^2) tells the caller when dt must shrink.
  * random numbers: oracle/philox.py stream layout.

Parity: pinned through its parts and through the statistical equivalence with
the expectation values of App. C (tests/test_oracle_mc.py).
"""
import numpy as np

from . import units
from .aniso import new_direction
from .kernel import overlap_g_vec
from .meanfield import pair_geometry
from .philox import bern_uniforms, dm_uniforms, pair_normals
from .xsec import family, sigma_of_v

NO_PARTNER = 0xFFFFFFFF


def pcap(m_chi, mu):
    """Right-hand side of Eq. prob_criterion."""
    return np.minimum(0.1, 1e-4 * ((m_chi + mu) / mu) ** 2)


def pair_probabilities(dm, gas, pi, pj, params, step, dt, g=None):
    """Per-pair (P_ij, v^B_ij, v_rel) with the pair's own Philox stream."""
    if g is None:
        d = pair_geometry(dm, gas, pi, pj, params["periodic"], params["box"])
        g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    z = pair_normals(params["seed"], step, dm["id"][pi].astype(np.uint64), gas["id"][pj].astype(np.uint64))
    s = np.sqrt(units.varsigma2_kms2(gas["T"][pj], gas["mu"][pj]))
    vB = gas["vel"][pj] + s[:, None] * z
    rel = dm["vel"][pi] - vB
    vrel = np.sqrt(np.sum(rel * rel, axis=1))
    sig = sigma_of_v(vrel, params)
    nB = gas["mass"][pj] * units.MSUN_PER_MP / gas["mu"][pj]
    P = nB * g * sig * vrel * dt
    return P, vB, vrel


def mc_scatter(dm, gas, pi, pj, params, step, dt, g=None):
    """Return a dict with vel_new[N_chi,3], scattered, partner (gas id), p_ratio_max,
    C_total, r, clamped, and for diagnostics the running-sum gap to r."""
    m_chi = params["m_chi_mp"]
    nd = len(dm["h"])
    P, vB, vrel = pair_probabilities(dm, gas, pi, pj, params, step, dt, g)
    r, cth, phi = dm_uniforms(params["seed"], step, dm["id"].astype(np.uint64))
    ratio = P / pcap(m_chi, gas["mu"][pj])
    p_ratio_max = np.zeros(nd)
    np.maximum.at(p_ratio_max, pi, ratio)

    order = np.lexsort((gas["id"][pj], pi))  # per DM, ascending gas id
    vel_new = dm["vel"].copy()
    scattered = np.zeros(nd, dtype=bool)
    partner = np.full(nd, NO_PARTNER, dtype=np.uint64)
    C_total = np.zeros(nd)
    clamped = np.zeros(nd, dtype=bool)
    gap = np.full(nd, np.inf)   # min_k |threshold - C_k| / C_k, for the boundary band
    starts = np.searchsorted(pi[order], np.arange(nd), side="left")
    ends = np.searchsorted(pi[order], np.arange(nd), side="right")
    for i in np.unique(pi):
        seg = order[starts[i]:ends[i]]
        C = np.cumsum(P[seg])                # sequential FP64 running sum
        C_total[i] = C[-1]
        thr = r[i]
        if C[-1] > 1.0:
            clamped[i] = True
            thr = r[i] * C[-1]
        gap[i] = np.min(np.abs(thr - C) / C)
        k = int(np.searchsorted(C, thr, side="right"))   # first k with thr < C_k
        if k >= seg.size:
            continue
        e = seg[k]
        j = pj[e]
        mu = gas["mu"][j]
        n_old = (dm["vel"][i] - vB[e]) / vrel[e]
        n_new = new_direction(n_old, cth[i], phi[i], params.get("beta", 0.0))
        vel_new[i] = dm["vel"][i] + mu / (m_chi + mu) * vrel[e] * (n_new - n_old)
        scattered[i] = True
        partner[i] = gas["id"][j]
    return dict(vel_new=vel_new, scattered=scattered, partner=partner, p_ratio_max=p_ratio_max,
                C_total=C_total, r=r, clamped=clamped, gap=gap, P=P, vB=vB, vrel=vrel)


def scatter_pair(v_chi, v_B, m_chi, m_B, n_new):
    """Eqs. scatter_chi and scatter_B for one collision (used by the conservation pin)."""
    rel = v_chi - v_B
    vrel = np.linalg.norm(rel)
    n_old = rel / vrel
    vc = v_chi + m_B / (m_chi + m_B) * vrel * (n_new - n_old)
    vb = v_B - m_chi / (m_chi + m_B) * vrel * (n_new - n_old)
    return vc, vb


def mc_scatter_bernoulli(dm, gas, pi, pj, params, step, dt, g=None, max_scatters=64):
    """The per-pair Bernoulli form in which Sec. 2.5 applies the Monte Carlo (the GIZMO
    implementation): the pairs of DM particle i, in ascending gas id, each scatter when
    r_ij < P_ij, where P_ij (Eq. dm-update-prob, with the pair's sample v^B_ij) is computed from
    the particle's velocity after any earlier scatter of the step, and the kick is Eq.
    scatter_chi with the pair's own isotropic direction.  r_ij and the direction come from the
    Bernoulli stream (oracle/philox.py); at most max_scatters scatters per particle.

    Returns the fields of mc_scatter (C_total and p_ratio_max at the start velocity, partner =
    the first partner) plus n_scatter, and gap = min over the tested pairs of |r_ij - P_ij| / P_ij."""
    m_chi = params["m_chi_mp"]
    nd = len(dm["h"])
    if g is None:
        d = pair_geometry(dm, gas, pi, pj, params["periodic"], params["box"])
        g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    P0, vB, _ = pair_probabilities(dm, gas, pi, pj, params, step, dt, g)
    r, cth, phi = bern_uniforms(params["seed"], step, dm["id"][pi].astype(np.uint64), gas["id"][pj].astype(np.uint64))
    ratio = P0 / pcap(m_chi, gas["mu"][pj])
    p_ratio_max = np.zeros(nd)
    np.maximum.at(p_ratio_max, pi, ratio)
    C_total = np.zeros(nd)
    np.add.at(C_total, pi, P0)
    nB = gas["mass"][pj] * units.MSUN_PER_MP / gas["mu"][pj]
    s0, v0, n = units.sigma_kpc2(params["sigma0_cm2"]), params["v0_kms"], params["n"]
    powerlaw = family(params) == "powerlaw"

    order = np.lexsort((gas["id"][pj], pi))
    starts = np.searchsorted(pi[order], np.arange(nd), side="left")
    ends = np.searchsorted(pi[order], np.arange(nd), side="right")
    vel_new = dm["vel"].copy()
    scattered = np.zeros(nd, dtype=bool)
    partner = np.full(nd, NO_PARTNER, dtype=np.uint64)
    n_scatter = np.zeros(nd, dtype=np.int64)
    gap = np.full(nd, np.inf)
    for i in np.unique(pi):
        v = dm["vel"][i].copy()
        for e in order[starts[i]:ends[i]]:
            rel = v - vB[e]
            vr = np.sqrt(rel @ rel)
            if powerlaw:
                P = nB[e] * g[e] * s0 * (vr / v0) ** n * vr * dt
            else:
                P = nB[e] * g[e] * float(sigma_of_v(vr, params)) * vr * dt
            if P > 0:
                gap[i] = min(gap[i], abs(r[e] - P) / P)
            if r[e] < P:
                j = pj[e]
                mu = gas["mu"][j]
                n_new = new_direction(rel / vr, cth[e], phi[e], params.get("beta", 0.0))
                v = v + mu / (m_chi + mu) * vr * (n_new - rel / vr)
                if not scattered[i]:
                    scattered[i] = True
                    partner[i] = gas["id"][j]
                n_scatter[i] += 1
                if n_scatter[i] == max_scatters:
                    break
        vel_new[i] = v
    return dict(vel_new=vel_new, scattered=scattered, partner=partner, p_ratio_max=p_ratio_max,
                C_total=C_total, n_scatter=n_scatter, gap=gap)
