"""Pins for the cross-section family beyond the power law (oracle/xsec.py): the screened law
sigma0 / (1 + (v / v_c)^2)^2 reduces to the closed forms of the n = 0 law (v_c -> infinity)
and of the n = -4 law (v >> v_c); the quadratures approach the cold limits; the Monte Carlo
with this sigma(v) matches on average the App. C expectations computed by quadrature; the
moment equations with it conserve momentum and energy."""
import math

import numpy as np
import pytest

from oracle import mbode as MB
from oracle import mc as M
from oracle import units
from oracle import xsec as X
from oracle.expect import expected_dm
from oracle.kernel import overlap_g_vec
from oracle.meanfield import pair_geometry, pair_rates
from oracle.pairs import pairs_bruteforce
from oracle.rates import A_closed_arr, B_closed_arr, R_closed_arr
from paper_2603_24688_gb300 import workloads as W


def _p(v_c, **kw):
    return dict(dict(sigma0_cm2=1e-26, n=0, v0_kms=100.0, xsec="screened", v_c_kms=v_c), **kw)


def test_sigma_at_the_knee_and_far_from_it():
    s0 = units.sigma_kpc2(1e-26)
    p = _p(50.0)
    assert X.sigma_of_v(50.0, p) == s0 / 4.0
    assert X.sigma_of_v(0.0, p) == s0
    assert abs(X.sigma_of_v(5e4, p) / (s0 * (50.0 / 5e4) ** 4) - 1.0) < 3e-6
    assert X.sigma_bar_of_v(50.0, dict(p, beta=0.6)) == pytest.approx(s0 / 4.0 * 0.8, rel=1e-15)
    with pytest.raises(ValueError):
        X.sigma_of_v(1.0, dict(p, xsec="nonsense"))


def test_large_knee_is_the_constant_cross_section():
    rng = np.random.default_rng(1)
    w = rng.uniform(0.0, 400.0, 40)
    w[0] = 0.0
    s2 = rng.uniform(20.0, 300.0, 40) ** 2
    p = _p(1e9)
    s0 = units.sigma_kpc2(1e-26)
    for got, ref in ((X.A_arr(w, s2, p), A_closed_arr(w, s2, s0, 100.0, 0)),
                     (X.B_arr(w, s2, p), B_closed_arr(w, s2, s0, 100.0, 0)),
                     (X.R_arr(w, s2, p), R_closed_arr(w, s2, s0, 100.0, 0))):
        assert np.max(np.abs(got / ref - 1.0)) < 1e-9


def test_small_knee_is_the_inverse_fourth_power():
    # for v >> v_c, sigma -> sigma0 v_c^4 / v^4: the n = -4 law with sigma0' = sigma0 (v_c / v0)^4;
    # the flat core below v_c changes A and B by O((v_c / varsigma)^2)
    rng = np.random.default_rng(2)
    w = rng.uniform(50.0, 400.0, 20)
    s2 = rng.uniform(100.0, 300.0, 20) ** 2
    v_c = 0.05
    p = _p(v_c)
    s0 = units.sigma_kpc2(1e-26) * (v_c / 100.0) ** 4
    # sigma = sigma_-4 (1 + v_c^2 / v^2)^-2 < sigma_-4: the screened rates lie below by about
    # 2 v_c^2 <v^-2>; for the n = -4 weighting that average grows like log(varsigma / v_c) / varsigma^2
    bound = 10.0 * v_c ** 2 / s2 * (1.0 + np.log(np.sqrt(s2) / v_c))
    for got, ref in ((X.A_arr(w, s2, p), A_closed_arr(w, s2, s0, 100.0, -4)),
                     (X.B_arr(w, s2, p), B_closed_arr(w, s2, s0, 100.0, -4))):
        assert np.all(got < ref)
        assert np.all(1.0 - got / ref < bound)


def test_cold_gas_limits():
    p = _p(80.0)
    w = np.array([30.0, 80.0, 250.0])
    sig = X.sigma_of_v(w, p)
    # varsigma = 0 takes the limits; a small varsigma approaches them
    assert np.array_equal(X.A_arr(w, 0.0, p), sig * w)
    assert np.array_equal(X.B_arr(w, 0.0, p), sig * w ** 3)
    assert np.max(np.abs(X.A_arr(w, (1e-3 * w) ** 2, p) / (sig * w) - 1.0)) < 1e-5
    assert np.max(np.abs(X.B_arr(w, (1e-3 * w) ** 2, p) / (sig * w ** 3) - 1.0)) < 1e-5
    assert np.max(np.abs(X.R_arr(w, (1e-3 * w) ** 2, p) / (sig * w) - 1.0)) < 1e-5


def test_power_law_path_is_unchanged():
    w = W.box_workload(n_dm=64, n_gas=64, L=1.0, seed=5, n=-2, T_gas=1e5)
    dm, gas, prm = w["dm"], w["gas"], w["params"]
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    g, ww, A, B = pair_rates(dm, gas, pi, pj, prm)
    wn = np.sqrt(np.sum(ww * ww, axis=1))
    s2 = units.varsigma2_kms2(gas["T"][pj], gas["mu"][pj])
    s0 = units.sigma_kpc2(prm["sigma0_cm2"])
    assert np.array_equal(A, A_closed_arr(wn, s2, s0, prm["v0_kms"], prm["n"]))
    assert np.array_equal(B, B_closed_arr(wn, s2, s0, prm["v0_kms"], prm["n"]))


def test_mc_mean_matches_the_quadrature_expectation():
    w = W.box_workload(n_dm=96, n_gas=96, L=1.0, seed=6, n=0, bulk_dm=(80.0, 0, 0), T_gas=1e5, dt=8e-4)
    dm, gas, dt = w["dm"], w["gas"], w["dt"]
    # sigma0 raised so that sum_j P_ij is about 0.1-0.25 with the screened law (no clamps)
    prm = dict(w["params"], xsec="screened", v_c_kms=60.0, sigma0_cm2=12.0 * w["params"]["sigma0_cm2"])
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    d = pair_geometry(dm, gas, pi, pj, True, prm["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    E_dv, E_dE, E_P = expected_dm(dm, gas, pi, pj, prm, dt, g)
    R = 300
    nd = len(dm["h"])
    s1 = np.zeros((nd, 3))
    s2 = np.zeros((nd, 3))
    se = np.zeros(R)
    nscat = 0
    for step in range(R):
        out = M.mc_scatter(dm, gas, pi, pj, prm, step, dt, g)
        assert not out["clamped"].any()
        dv = out["vel_new"] - dm["vel"]
        s1 += dv
        s2 += dv * dv
        se[step] = (0.5 * dm["mass"] * (np.sum(out["vel_new"] ** 2, 1) - np.sum(dm["vel"] ** 2, 1))).sum()
        nscat += out["scattered"].sum()
    mean = s1 / R
    var = s2 / R - mean ** 2
    ok = var[:, 0] > 0
    zz = ((mean - E_dv)[ok] / np.sqrt(var[ok] / R)).reshape(-1)
    assert abs(np.mean(zz)) < 5 / math.sqrt(zz.size)
    assert 0.8 < np.median(np.abs(zz)) / 0.6745 < 1.2
    tot = (dm["mass"][:, None] * s1).sum(0) / R
    tot_err = np.sqrt((dm["mass"][:, None] ** 2 * var).sum(0) / R)
    assert np.all(np.abs(tot - (dm["mass"][:, None] * E_dv).sum(0)) < 5 * tot_err)
    lam = E_P.sum() * R
    assert lam > 500
    assert abs(nscat - lam) < 5 * math.sqrt(lam)
    assert abs(se.mean() - E_dE.sum()) < 0.05 * abs(E_dE.sum()) + 5 * se.std() / math.sqrt(R)


def test_moment_equations_with_the_screened_law():
    y0 = [200.0, 0.0, MB.theta_from_T(1e6, 2.0), MB.theta_from_T(1e4, 1.0)]
    p = MB.params(2.0, 1.0, 1e10, 1e10, 1e-26, 0, v_c_kms=150.0)
    _, ys = MB.integrate(y0, p, 1.0, 100)
    P, E = MB.momentum(ys, p), MB.energy(ys, p)
    assert np.max(np.abs(P / P[0] - 1)) < 1e-13
    assert np.max(np.abs(E / E[0] - 1)) < 1e-8
    # slower than the constant cross section it tends to for v_c -> infinity
    p0 = MB.params(2.0, 1.0, 1e10, 1e10, 1e-26, 0)
    _, y_flat = MB.integrate(y0, p0, 1.0, 100)
    _, y_big = MB.integrate(y0, MB.params(2.0, 1.0, 1e10, 1e10, 1e-26, 0, v_c_kms=1e9), 1.0, 20)
    assert ys[-1, 0] > y_flat[-1, 0] + 5.0
    assert abs(y_big[-1, 0] - y_flat[::5][-1, 0]) < 1e-3
