"""Physical constants and the code-unit system used by the oracle.

Code units: length kpc, velocity km/s, mass Msun, time kpc/(km/s).  Temperatures
are in K and particle masses (m_chi, mu_j) in units of the proton mass m_p.
The paper works with k_B = 1 and writes the gas Maxwellian as G(v - V, T/mu)
(Eq. macroparticle-DF_B); here the 1D velocity variance is
varsigma^2 = k_B T / (mu m_p), expressed in (km/s)^2.

The cross section is sigma(v) = sigma0 (v / v0)^n (Sec. 2.4 writes v0 = c; any
reference speed v0 is the same law with sigma0' = sigma0 (v0/c)^n).
"""

K_B_CGS = 1.380649e-16          # erg / K (exact, SI 2019)
M_P_G = 1.67262192369e-24       # proton mass [g] (CODATA 2018)
KPC_CM = 3.0856775814913673e21  # kpc [cm]
MSUN_G = 1.98841e33             # solar mass [g]
KM_CM = 1.0e5                   # km [cm]

# Number of particles of mass 1 m_p in one Msun.
MSUN_PER_MP = MSUN_G / M_P_G


def varsigma2_kms2(T_K, mu_mp):
    """1D thermal velocity variance k_B T / (mu m_p) in (km/s)^2."""
    return K_B_CGS * T_K / (mu_mp * M_P_G) / (KM_CM * KM_CM)


def sigma_kpc2(sigma_cm2):
    """Cross section converted from cm^2 to kpc^2."""
    return sigma_cm2 / (KPC_CM * KPC_CM)


def u_from_T(T_K, mu_mp):
    """Specific thermal energy u = (3/2) k_B T / mu in (km/s)^2."""
    return 1.5 * varsigma2_kms2(T_K, mu_mp)


def T_from_u(u_kms2, mu_mp):
    """Inverse of u_from_T."""
    return u_kms2 * (KM_CM * KM_CM) * mu_mp * M_P_G / (1.5 * K_B_CGS)
