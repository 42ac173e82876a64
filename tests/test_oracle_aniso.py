"""Pins for the anisotropic scattering family dsigma/dOmega ~ 1 + beta cos theta
(oracle/aniso.py): the sampled cosine inverts the closed-form distribution, its moments are
those of the density, the new direction is a unit vector at the drawn angle to the old one,
and the Monte Carlo (total sigma, anisotropic angles) matches on average the App. C
expectations taken with the momentum-transfer cross section sigma (1 - beta / 3) (Sec. 2.4),
not those with sigma."""
import math

import numpy as np
import pytest

from oracle import aniso as A
from oracle import mc as M
from oracle.expect import expected_dm
from oracle.kernel import overlap_g_vec
from oracle.meanfield import pair_geometry
from oracle.pairs import pairs_bruteforce
from paper_2603_24688_gb300 import workloads as W

BETAS = [-1.0, -0.6, 0.3, 0.9, 1.0]


@pytest.mark.parametrize("beta", BETAS)
def test_sampled_cosine_inverts_the_distribution(beta):
    c = np.linspace(-1.0, 1.0, 20001)
    m = A.cos_from_isotropic(c, beta)
    assert np.all(np.abs(m) <= 1.0 + 1e-15)
    assert np.all(np.diff(m) >= 0.0)                       # a quantile function is monotone
    # F(m) = u with u = (c + 1) / 2, the isotropic draw's quantile
    assert np.max(np.abs(A.cdf(m, beta) - 0.5 * (c + 1.0))) < 1e-14
    assert A.cdf(-1.0, beta) == 0.0 and abs(A.cdf(1.0, beta) - 1.0) < 1e-15


def test_zero_beta_is_the_isotropic_draw():
    c = np.linspace(-1.0, 1.0, 1001)
    assert np.array_equal(A.cos_from_isotropic(c, 0.0), c)
    assert A.sbar_factor(0.0) == 1.0


@pytest.mark.parametrize("beta", BETAS)
def test_moments_of_the_sampled_cosine(beta):
    # midpoint quadrature over the quantile u: <m> = beta / 3, <m^2> = 1 / 3 for this density
    u = (np.arange(400000) + 0.5) / 400000
    m = A.cos_from_isotropic(2.0 * u - 1.0, beta)
    assert abs(m.mean() - beta / 3.0) < 1e-6
    assert abs((m * m).mean() - 1.0 / 3.0) < 1e-6
    assert abs(A.sbar_factor(beta) - (1.0 - m.mean())) < 1e-6


def test_new_direction_is_a_unit_vector_at_the_drawn_angle():
    rng = np.random.default_rng(4)
    ns = rng.normal(size=(2000, 3))
    ns /= np.linalg.norm(ns, axis=1)[:, None]
    ns[:4] = [[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, -1.0, 0]]   # the basis' special cases
    for k, n in enumerate(ns):
        e1, e2 = A.onb(n)
        B = np.array([e1, e2, n])
        assert np.max(np.abs(B @ B.T - np.eye(3))) < 1e-12
        beta = BETAS[k % len(BETAS)]
        c, phi = rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
        n2 = A.new_direction(n, c, phi, beta)
        assert abs(np.linalg.norm(n2) - 1.0) < 1e-12
        assert abs(n2 @ n - A.cos_from_isotropic(c, beta)) < 1e-12
        # the azimuth is measured in (e1, e2)
        assert abs(math.atan2(n2 @ e2, n2 @ e1) % (2 * np.pi) - phi % (2 * np.pi)) < 1e-9 or \
            abs(1.0 - abs(n2 @ n)) < 1e-9


def test_out_of_range_beta_is_refused():
    for b in (-1.5, 1.0000001, float("nan")):
        with pytest.raises(ValueError):
            A.check_beta(b)


@pytest.mark.parametrize("beta", [0.9, -0.6])
def test_mc_mean_matches_the_momentum_transfer_expectation(beta):
    # 192 DM + 192 gas in a periodic box with a bulk DM drift; App. C expectations with
    # sigma_bar = sigma (1 - beta / 3), while the scatter count follows the total sigma
    w = W.box_workload(n_dm=192, n_gas=192, L=1.0, seed=3, n=0, bulk_dm=(80.0, 0, 0), T_gas=1e5, dt=8e-4)
    dm, gas, dt = w["dm"], w["gas"], w["dt"]
    prm = dict(w["params"], beta=beta)
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    d = pair_geometry(dm, gas, pi, pj, True, prm["box"])
    g = overlap_g_vec(d, dm["h"][pi], gas["h"][pj])
    E_dv, E_dE, E_P = expected_dm(dm, gas, pi, pj, prm, dt, g)
    E_dv_iso, _, E_P_iso = expected_dm(dm, gas, pi, pj, dict(prm, beta=0.0), dt, g)
    assert np.allclose(E_P, E_P_iso)                       # the probability takes sigma
    assert np.allclose(E_dv, A.sbar_factor(beta) * E_dv_iso)
    R = 300
    nd = len(dm["h"])
    s1 = np.zeros((nd, 3))
    s2 = np.zeros((nd, 3))
    se = np.zeros(R)
    nscat = 0
    for step in range(R):
        out = M.mc_scatter(dm, gas, pi, pj, prm, step, dt, g)
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
    want = (dm["mass"][:, None] * E_dv).sum(0)
    assert abs(tot[0] - want[0]) < 5 * tot_err[0]
    # ... and not the isotropic expectation: the drift's momentum transfer differs by beta / 3
    iso = (dm["mass"][:, None] * E_dv_iso).sum(0)
    assert abs(tot[0] - iso[0]) > 5 * tot_err[0]
    lam = E_P.sum() * R
    assert abs(nscat - lam) < 5 * math.sqrt(lam)
    assert abs(se.mean() - E_dE.sum()) < 0.05 * abs(E_dE.sum()) + 5 * se.std() / math.sqrt(R)
