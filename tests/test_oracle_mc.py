"""Pins for the oracle's DM Monte Carlo (Eqs. dm-update-*, scatter_chi/B; App. C)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import mc as M
from oracle import units
from oracle.expect import expected_dm
from oracle.kernel import overlap_g_vec
from oracle.meanfield import pair_geometry
from oracle.pairs import pairs_bruteforce
from paper_2603_24688_gb300 import workloads as W


def test_single_scatter_conserves_momentum_energy_and_speed():
    # Eqs. scatter_chi and scatter_B: m_chi dv_chi + m_B dv_B = 0, |v_rel| and kinetic energy kept
    rng = np.random.default_rng(0)
    for _ in range(50):
        vc, vb = rng.normal(0, 100, 3), rng.normal(0, 30, 3)
        mc, mb = rng.uniform(0.1, 10), rng.uniform(0.5, 4)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        vc2, vb2 = M.scatter_pair(vc, vb, mc, mb, n)
        p0, p1 = mc * vc + mb * vb, mc * vc2 + mb * vb2
        e0 = 0.5 * mc * vc @ vc + 0.5 * mb * vb @ vb
        e1 = 0.5 * mc * vc2 @ vc2 + 0.5 * mb * vb2 @ vb2
        assert np.allclose(p0, p1, rtol=0, atol=1e-11 * np.abs(p0).max())
        assert abs(e1 - e0) < 1e-12 * e0
        assert abs(np.linalg.norm(vc2 - vb2) - np.linalg.norm(vc - vb)) < 1e-12 * np.linalg.norm(vc - vb)
        assert np.allclose((vc2 - vb2) / np.linalg.norm(vc2 - vb2), n, atol=1e-12)


def test_probability_cold_gas_reduces_to_n_sigma_v_dt():
    # with T_j = 0 the sampled v^B equals V_j, so P_ij = (M_j/mu_j) g sigma(w) w dt exactly
    w = W.box_workload(n_dm=64, n_gas=64, seed=3, n=-2)
    w["gas"]["T"][:] = 0.0
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    P, vB, vrel = M.pair_probabilities(w["dm"], w["gas"], pi, pj, w["params"], 0, w["dt"])
    d = pair_geometry(w["dm"], w["gas"], pi, pj, True, w["params"]["box"])
    g = overlap_g_vec(d, w["dm"]["h"][pi], w["gas"]["h"][pj])
    wv = np.linalg.norm(w["dm"]["vel"][pi] - w["gas"]["vel"][pj], axis=1)
    sig = units.sigma_kpc2(1e-24) * (wv / 100.0) ** -2
    ref = w["gas"]["mass"][pj] * units.MSUN_PER_MP / w["gas"]["mu"][pj] * g * sig * wv * w["dt"]
    np.testing.assert_allclose(P, ref, rtol=1e-13)


def _small_box(n=0, seed=21):
    # 192 DM + 192 gas in a periodic box, dt raised so that sum_j P_ij ~ 0.2
    w = W.box_workload(n_dm=192, n_gas=192, L=1.0, seed=seed, n=n, bulk_dm=(80.0, 0, 0),
                       T_gas=1e5, dt=8e-4)
    return w


@pytest.mark.parametrize("n", [0, -2])
def test_mc_mean_matches_expectation(n):
    # App. C: averaged over realisations, each DM particle's velocity change converges to
    # E[dv_i]; per-particle z-scores are standard normal and the scatter count matches
    # sum_j E[P_ij] (n > -4)
    w = _small_box(n)
    dm, gas, prm, dt = w["dm"], w["gas"], w["params"], w["dt"]
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    d = pair_geometry(dm, gas, pi, pj, True, prm["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    E_dv, E_dE, E_P = expected_dm(dm, gas, pi, pj, prm, dt, g)
    R = 300
    nd = len(dm["h"])
    s1 = np.zeros((nd, 3))
    s2 = np.zeros((nd, 3))
    se1 = np.zeros(nd)
    nscat = 0
    Ctot = []
    for step in range(R):
        out = M.mc_scatter(dm, gas, pi, pj, prm, step, dt, g)
        assert not out["clamped"].any()
        dv = out["vel_new"] - dm["vel"]
        s1 += dv
        s2 += dv * dv
        se1 += 0.5 * dm["mass"] * (np.sum(out["vel_new"] ** 2, 1) - np.sum(dm["vel"] ** 2, 1))
        nscat += out["scattered"].sum()
        Ctot.append(out["C_total"])
    mean = s1 / R
    var = s2 / R - mean ** 2
    ok = var[:, 0] > 0
    z = (mean - E_dv)[ok] / np.sqrt(var[ok] / R)
    zz = z.reshape(-1)
    # per-particle z-scores ~ N(0, 1); heavy tails are trimmed by the robust scale check
    assert abs(np.mean(zz)) < 5 / math.sqrt(zz.size)
    assert 0.8 < np.median(np.abs(zz)) / 0.6745 < 1.2
    # the global momentum change converges to sum_i M_i E[dv_i]
    tot = (dm["mass"][:, None] * s1).sum(0) / R
    tot_err = np.sqrt((dm["mass"][:, None] ** 2 * var).sum(0) / R)
    assert np.all(np.abs(tot - (dm["mass"][:, None] * E_dv).sum(0)) < 5 * tot_err)
    # expected number of scatters: sum over DM of the averaged probability
    lam = E_P.sum() * R
    assert abs(nscat - lam) < 5 * math.sqrt(lam)
    # energy: mean realised change vs App. C expectation (global)
    e_mean = se1.sum() / R
    assert abs(e_mean - E_dE.sum()) < 0.05 * abs(E_dE.sum()) + 5 * np.std(se1) / math.sqrt(R)


def test_partner_choice_follows_probabilities():
    # the categorical draw picks partner j with probability P_ij (given the draws), tested by
    # recomputing each step's P and comparing chosen-partner frequencies with sum P_ij / sum C
    w = _small_box(0, seed=5)
    dm, gas, prm, dt = w["dm"], w["gas"], w["params"], w["dt"]
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    d = pair_geometry(dm, gas, pi, pj, True, prm["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    i0 = np.bincount(pi).argmax()
    sel = pi == i0
    exp_counts = np.zeros(sel.sum())
    obs_counts = np.zeros(sel.sum())
    ids = gas["id"][pj[sel]]
    for step in range(400):
        out = M.mc_scatter(dm, gas, pi, pj, prm, step, dt, g)
        exp_counts += out["P"][sel]
        if out["scattered"][i0]:
            obs_counts[np.nonzero(ids == out["partner"][i0])[0][0]] += 1
    total_exp = exp_counts.sum()
    assert abs(obs_counts.sum() - total_exp) < 5 * math.sqrt(total_exp)
    # pool into 4 bins of equal expected count and chi^2-test the shape
    order = np.argsort(exp_counts)
    cum = np.cumsum(exp_counts[order]) / total_exp
    bins = np.minimum((cum * 4).astype(int), 3)
    o = np.bincount(bins, weights=obs_counts[order], minlength=4)
    e = np.bincount(bins, weights=exp_counts[order], minlength=4) * obs_counts.sum() / total_exp
    chi2 = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, 3) > 1e-4


@pytest.mark.parametrize("n,beta", [(0, 0.0), (-2, 0.0), (0, 0.9)])
def test_bernoulli_variant_mean_matches_expectation(n, beta):
    # the per-pair Bernoulli form has the same expectation (App. C) as the categorical draw to
    # first order in P (a scatter changes the later probabilities only at second order); with
    # anisotropic angles (beta != 0) the expectation takes sigma_bar = sigma (1 - beta / 3)
    w = _small_box(n)
    dm, gas, dt = w["dm"], w["gas"], w["dt"]
    prm = dict(w["params"], beta=beta)
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    d = pair_geometry(dm, gas, pi, pj, True, prm["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    E_dv, E_dE, E_P = expected_dm(dm, gas, pi, pj, prm, dt, g)
    R = 300
    nd = len(dm["h"])
    s1 = np.zeros((nd, 3))
    s2 = np.zeros((nd, 3))
    nscat = 0
    for step in range(R):
        out = M.mc_scatter_bernoulli(dm, gas, pi, pj, prm, step, dt, g)
        dv = out["vel_new"] - dm["vel"]
        s1 += dv
        s2 += dv * dv
        nscat += out["n_scatter"].sum()
    mean = s1 / R
    var = s2 / R - mean ** 2
    ok = var[:, 0] > 0
    zz = ((mean - E_dv)[ok] / np.sqrt(var[ok] / R)).reshape(-1)
    assert abs(np.mean(zz)) < 5 / math.sqrt(zz.size)
    assert 0.8 < np.median(np.abs(zz)) / 0.6745 < 1.2
    lam = E_P.sum() * R
    assert abs(nscat - lam) < 5 * math.sqrt(lam) + 0.05 * lam


def test_bernoulli_variant_extremes():
    # dt -> 0: nothing scatters.  dt huge: the first scatter is the smallest gas id whose r_ij is
    # below its P_ij at the start velocity (a pair at the edge of the kernel, where g is tiny,
    # can still miss), later scatters are capped, and a particle whose only pair scatters keeps
    # its speed relative to that pair's gas sample
    from oracle.philox import bern_uniforms
    w = _small_box(0)
    dm, gas, prm = w["dm"], w["gas"], w["params"]
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    none = M.mc_scatter_bernoulli(dm, gas, pi, pj, prm, 3, 1e-30)
    assert not none["scattered"].any() and np.array_equal(none["vel_new"], dm["vel"])
    dt = 1e6
    allp = M.mc_scatter_bernoulli(dm, gas, pi, pj, prm, 3, dt, max_scatters=8)
    P0, vB, vrel = M.pair_probabilities(dm, gas, pi, pj, prm, 3, dt)
    r, _, _ = bern_uniforms(prm["seed"], 3, dm["id"][pi].astype(np.uint64), gas["id"][pj].astype(np.uint64))
    counts = np.bincount(pi, minlength=len(dm["h"]))
    assert np.all(allp["n_scatter"] <= np.minimum(counts, 8))
    assert np.count_nonzero(allp["n_scatter"] == 8) > 0
    for i in np.unique(pi):
        hit = (pi == i) & (r < P0)
        want = gas["id"][pj[hit]].min() if hit.any() else M.NO_PARTNER
        assert allp["partner"][i] == want
    for i in np.nonzero(counts == 1)[0][:10]:
        e = np.nonzero(pi == i)[0][0]
        if allp["scattered"][i]:
            assert abs(np.linalg.norm(allp["vel_new"][i] - vB[e]) - vrel[e]) < 1e-9 * vrel[e]
