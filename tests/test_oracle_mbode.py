"""Pins for the naive Maxwell-Boltzmann prediction of the periodic-box tests (oracle/mbode.py):
its conservation laws, its fixed point, a brute-force Monte Carlo of isotropic collisions
between two Maxwellian populations (which fixes the re-derived temperature equations, with
m_chi != m_B), and the Jarque-Bera statistic on samples of known skewness and kurtosis."""
import numpy as np
import pytest

from oracle import mbode as M
from oracle.units import MSUN_PER_MP, sigma_kpc2


def _fiducial(n=0, sigma0=1e-26, m_chi=2.0, m_B=1.0):
    return M.params(m_chi, m_B, 1e10, 1e10, sigma0, n)


def test_momentum_and_energy_are_conserved():
    for n, s0 in ((0, 1e-26), (-2, 2e-33), (-4, 5e-40)):
        p = _fiducial(n, s0)
        y0 = [200.0, 0.0, M.theta_from_T(1e6, 2.0), M.theta_from_T(1e4, 1.0)]
        _, ys = M.integrate(y0, p, 1.0, 200)
        P, E = M.momentum(ys, p), M.energy(ys, p)
        assert np.max(np.abs(P / P[0] - 1)) < 1e-13
        # RK4 conserves the linear momentum exactly; the energy to its truncation error, which
        # falls as h^4: halving h cuts the drift by about 16
        d1 = abs(E[-1] / E[0] - 1)
        _, ys2 = M.integrate(y0, p, 1.0, 400)
        d2 = abs(M.energy(ys2, p)[-1] / E[0] - 1)
        assert d1 < 1e-8 and (d2 < d1 / 8 or d1 < 1e-13), (n, d1, d2)


def test_equilibrium_is_a_fixed_point_and_is_approached():
    p = _fiducial()
    T = 3e5
    y = np.array([50.0, 50.0, M.theta_from_T(T, 2.0), M.theta_from_T(T, 1.0)])
    assert np.max(np.abs(M.rhs(y, p))) < 1e-12 * max(1.0, np.max(np.abs(y)))
    _, ys = M.integrate([200.0, 0.0, M.theta_from_T(1e6, 2.0), M.theta_from_T(1e4, 1.0)], p, 6.0, 600)
    Tc, Tb = M.T_from_theta(ys[-1, 2], 2.0), M.T_from_theta(ys[-1, 3], 1.0)
    assert abs(ys[-1, 0] - ys[-1, 1]) < 0.5 and abs(Tc / Tb - 1) < 1e-2
    # the common bulk velocity is the momentum-weighted mean, here (200 + 0) / 2
    assert abs(ys[-1, 0] - 100.0) < 0.5


@pytest.mark.parametrize("m_chi,m_B,n,sig0,V,Tc,Tb", [
    (2.0, 1.0, 0, 1e-26, 200.0, 1e6, 1e4),
    (10.0, 0.6, 0, 1e-26, 120.0, 5e6, 3e5),
    (0.5, 1.0, -2, 2e-33, 80.0, 2e4, 4e5),
])
def test_rates_against_monte_carlo_collisions(m_chi, m_B, n, sig0, V, Tc, Tb):
    """Sample chi and B velocities from their Maxwellians, weight each pair by the collision
    rate n_B sigma(u) u, scatter isotropically in the centre-of-mass frame and average the
    changes of the chi bulk velocity and of its 3 theta / 2; likewise for B."""
    p = M.params(m_chi, m_B, 1e10, 2e10, sig0, n)
    rng = np.random.default_rng(17)
    N = 2_000_000
    tc, tb = M.theta_from_T(Tc, m_chi), M.theta_from_T(Tb, m_B)
    vc = rng.normal(0.0, np.sqrt(tc), (N, 3))
    vc[:, 0] += V
    vb = rng.normal(0.0, np.sqrt(tb), (N, 3))
    u = vc - vb
    un = np.linalg.norm(u, axis=1)
    sig = sigma_kpc2(sig0) * (un / 100.0) ** n
    nhat = rng.normal(size=(N, 3))
    nhat /= np.linalg.norm(nhat, axis=1)[:, None]
    mt = m_chi + m_B
    dvc = (m_B / mt) * (un[:, None] * nhat - u)           # Delta v_chi; Delta v_B = -(m_chi/m_B) dvc
    dvb = -(m_chi / m_B) * dvc
    nB = 2e10 * MSUN_PER_MP / m_B                           # number densities per kpc^3
    nc = 1e10 * MSUN_PER_MP / m_chi
    wgt = sig * un
    # per particle: d<v>/dt = n_other <sigma u Delta v>; d<v^2/2>/dt likewise
    rate_vc = nB * wgt[:, None] * dvc
    rate_ec = nB * wgt * 0.5 * (np.sum((vc + dvc) ** 2, 1) - np.sum(vc ** 2, 1))
    rate_vb = nc * wgt[:, None] * dvb
    rate_eb = nc * wgt * 0.5 * (np.sum((vb + dvb) ** 2, 1) - np.sum(vb ** 2, 1))
    dVc, dVb = rate_vc[:, 0].mean(), rate_vb[:, 0].mean()
    # d theta/dt = (2/3) (d<v^2/2>/dt - V dV/dt)
    dtc = (2.0 / 3.0) * (rate_ec.mean() - V * dVc)
    dtb = (2.0 / 3.0) * (rate_eb.mean() - 0.0 * dVb)
    ref = M.rhs(np.array([V, 0.0, tc, tb]), p)
    errs = [rate_vc[:, 0].std(), rate_vb[:, 0].std(), (2 / 3) * rate_ec.std(), (2 / 3) * rate_eb.std()]
    for k, (got, want, sd) in enumerate(zip([dVc, dVb, dtc, dtb], ref, errs)):
        assert abs(got - want) < 5.0 * sd / np.sqrt(N) + 1e-12 * abs(want), (k, got, want, sd / np.sqrt(N))


def test_jarque_bera_on_known_samples():
    rng = np.random.default_rng(3)
    assert M.jarque_bera(rng.standard_normal(2_000_000)) < 1e-4
    # uniform: S = 0, K = 9/5, so JB = (6/5)^2 / 24 = 0.06
    assert abs(M.jarque_bera(rng.uniform(size=2_000_000)) - 0.06) < 2e-3
    # exponential: S = 2, K = 9, JB = (4 + 9) / 6
    assert abs(M.jarque_bera(rng.exponential(size=4_000_000)) - 13.0 / 6.0) < 0.15
