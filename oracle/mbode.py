"""The naive Maxwell-Boltzmann prediction of the periodic-box tests (oracle, FP64; test
infrastructure: only tests/ use it).

App. F: if both species stay Maxwellian, each is described by its bulk velocity V and its
temperature, and the first two moments of the Boltzmann equation give four ODEs.  With both
bulk velocities along x they read, in velocity-squared temperatures theta = k_B T / m
(so v_th^2 = theta_chi + theta_B) and V = |V_chi - V_B|:

    dV_chi/dt         = F_B   A(V; v_th^2) (V_B - V_chi)
    dV_B/dt           = F_chi A(V; v_th^2) (V_chi - V_B)
    (3/2) dtheta_chi/dt = (F_B / v_th^2)   [B (m_B theta_B - m_chi theta_chi) / (m_chi + m_B) + A theta_chi V^2]
    (3/2) dtheta_B/dt   = (F_chi / v_th^2) [B (m_chi theta_chi - m_B theta_B) / (m_chi + m_B) + A theta_B V^2]

with F_s = rho_s / (m_chi + m_B) (a number density times the mass ratio, in code units
rho_s Msun/m_p / (m_chi + m_B) per kpc^3) and A, B the integrals of Eqs. scrA/scrB at the
relative velocity V and variance v_th^2.

Reading: App. F prints the left sides of the temperature equations as dT/dt.  Multiplied out
(T = m theta), the right sides above are those of App. F; the left side that makes them the
moments of the collision term is (3 / 2m) dT/dt, the form of Eq. gas-dTdt.  Derivation (isotropic
sigma_bar; per chi particle, relative velocity u ~ N(V, v_th^2), centre-of-mass velocity
v_cm with E[v_cm | u] = V_cm + (T_chi - T_B)/((m_chi + m_B) v_th^2) (u - V)): the momentum
rate is -n_B mu_red <sigma u u> = -n_B mu_red A V, the energy rate -n_B mu_red <sigma u v_cm.u>,
and subtracting the bulk part leaves the temperature equation above.  Momentum
rho_chi V_chi + rho_B V_B and energy sum_s rho_s (V_s^2/2 + 3 theta_s / 2) are conserved
exactly by these equations (tests/test_oracle_mbode.py).

The integrator is the classical fourth-order Runge-Kutta method with a fixed step.
"""
import numpy as np

from .aniso import sbar_factor
from .rates import A_closed, A_quad, B_closed, B_quad
from .units import MSUN_PER_MP, sigma_kpc2, varsigma2_kms2
from .xsec import sigma_bar_of_v


def params(m_chi, m_B, rho_chi, rho_B, sigma0_cm2, n, v0_kms=100.0, beta=0.0, v_c_kms=None):
    """Constants of the ODE in code units (kpc, km/s, Msun; masses in m_p).  The moment
    equations take the momentum-transfer cross section: sigma0 (1 - beta / 3) for
    dsigma/dOmega proportional to 1 + beta cos theta (oracle/aniso.py).  v_c_kms selects the
    screened law sigma0 / (1 + (v / v_c)^2)^2 instead of the power law (oracle/xsec.py); A and
    B are then taken by quadrature."""
    ratio = MSUN_PER_MP
    sbar_fn = None
    if v_c_kms is not None:
        xp = dict(xsec="screened", sigma0_cm2=float(sigma0_cm2), v_c_kms=float(v_c_kms), beta=beta)
        sbar_fn = lambda u: float(sigma_bar_of_v(u, xp))
    return dict(m_chi=float(m_chi), m_B=float(m_B), n=int(n), v0=float(v0_kms), sbar_fn=sbar_fn,
                sigma0=sigma_kpc2(float(sigma0_cm2)) * sbar_factor(beta),
                F_chi=float(rho_chi) * ratio / (m_chi + m_B), F_B=float(rho_B) * ratio / (m_chi + m_B),
                rho_chi=float(rho_chi), rho_B=float(rho_B))


def theta_from_T(T_kelvin, m_mp):
    """k_B T / m in (km/s)^2."""
    return varsigma2_kms2(np.asarray(T_kelvin, dtype=np.float64), m_mp)


def T_from_theta(theta, m_mp):
    return np.asarray(theta, dtype=np.float64) / varsigma2_kms2(1.0, m_mp)


def rhs(y, p):
    """Derivatives of y = (V_chi, V_B, theta_chi, theta_B)."""
    Vc, Vb, tc, tb = y
    vth2 = tc + tb
    V = abs(Vc - Vb)
    if p.get("sbar_fn") is not None:                 # quadrature; V = 0 read at 1e-9 v_th
        Vq = max(V, 1e-9 * np.sqrt(vth2))
        A = A_quad(Vq, vth2, p["sbar_fn"])
        B = B_quad(Vq, vth2, p["sbar_fn"])
    else:
        A = A_closed(V, vth2, p["sigma0"], p["v0"], p["n"])
        B = B_closed(V, vth2, p["sigma0"], p["v0"], p["n"])
    mc, mb = p["m_chi"], p["m_B"]
    dVc = p["F_B"] * A * (Vb - Vc)
    dVb = p["F_chi"] * A * (Vc - Vb)
    heat = B * (mb * tb - mc * tc) / (mc + mb)
    dtc = (2.0 / 3.0) * p["F_B"] / vth2 * (heat + A * tc * V * V)
    dtb = (2.0 / 3.0) * p["F_chi"] / vth2 * (-heat + A * tb * V * V)
    return np.array([dVc, dVb, dtc, dtb])


def integrate(y0, p, t_end, nsteps):
    """RK4 from t = 0 to t_end in nsteps equal steps; returns (t [nsteps+1], y [nsteps+1, 4])."""
    h = t_end / nsteps
    ys = np.empty((nsteps + 1, 4))
    ys[0] = y = np.asarray(y0, dtype=np.float64)
    for k in range(nsteps):
        k1 = rhs(y, p)
        k2 = rhs(y + 0.5 * h * k1, p)
        k3 = rhs(y + 0.5 * h * k2, p)
        k4 = rhs(y + h * k3, p)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        ys[k + 1] = y
    return np.linspace(0.0, t_end, nsteps + 1), ys


def momentum(y, p):
    return p["rho_chi"] * y[..., 0] + p["rho_B"] * y[..., 1]


def energy(y, p):
    return (p["rho_chi"] * (0.5 * y[..., 0] ** 2 + 1.5 * y[..., 2])
            + p["rho_B"] * (0.5 * y[..., 1] ** 2 + 1.5 * y[..., 3]))


def jarque_bera(v):
    """JB = [S^2 + (K - 3)^2 / 4] / 6 of a sample, without the factor N (App. F)."""
    v = np.asarray(v, dtype=np.float64)
    d = v - v.mean()
    m2 = np.mean(d * d)
    S = np.mean(d ** 3) / m2 ** 1.5
    K = np.mean(d ** 4) / (m2 * m2)
    return (S * S + 0.25 * (K - 3.0) ** 2) / 6.0
