"""Periodic-box relaxation runs of the App. F test problem, stepped by the library.

A run repeats the interaction step (`dmb_step`: pairs, mean field on the gas, Monte Carlo on the
dark matter, kicks) followed by a drift x += v dt of both species, wrapped into the box; gravity
and hydrodynamics are off, as in the test problem.  Every `snap` steps it records, from the
device state:

* the bulk velocities along x of both species (mass-weighted means);
* the dark-matter temperature from its velocity dispersion, theta_chi = k_B T_chi / m_chi;
* the gas temperature: the internal one plus the dispersion of the gas particles' own
  velocities (the gas particles receive slightly different kicks; with hydrodynamics off that
  spread stays kinetic, and the two together are the gas temperature the moment equations
  describe);
* total momentum along x and total energy (kinetic plus gas internal plus dark-matter thermal
  is all kinetic for the particles);
* the Jarque-Bera statistic of the dark-matter velocities along each axis (App. F, without
  the factor N).

`ROWS` holds Table test_params (App. F): the fiducial test, the rows that vary one setting, and
the recreation of the test of Fischer et al. 2025, Sec. 3.4 (the table's last row).
Cross sections of the rows with n != 0 are quoted at v0 = c, as the paper writes sigma(v).
The table gives neither the box side nor the gas molecular weight: runs use L = 1 kpc and
mu = 1 unless told otherwise.
"""
import time

import numpy as np

from . import dmb
from . import workloads as W

C_KMS = 299792.458
GEV_PER_MP = 0.93827208816
KB_OVER_MP = 1.380649e-16 / 1.67262192369e-24 / 1e10     # k_B / m_p in (km/s)^2 / K

# name -> (m_chi [m_p], sigma0 [cm^2], n, V_chi0 [km/s], T_chi0 [K], T_B0 [K],
#          rho_chi, rho_B [Msun / kpc^3], N_chi, N_B)
ROWS = {
    "fiducial": (2.0, 1e-26, 0, 200.0, 1e6, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "V_chi=0": (2.0, 1e-26, 0, 0.0, 1e6, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "T_chi=T_B=0": (2.0, 1e-26, 0, 200.0, 1e1, 1e1, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "rho_B=10rho_chi": (2.0, 1e-26, 0, 200.0, 1e6, 1e4, 1e9, 1e10, 32 ** 3, 32 ** 3),
    "rho_chi=10rho_B": (2.0, 1e-26, 0, 200.0, 1e6, 1e4, 1e10, 1e9, 32 ** 3, 32 ** 3),
    "N_chi=24^3": (2.0, 1e-26, 0, 200.0, 1e6, 1e4, 1e10, 1e10, 24 ** 3, 32 ** 3),
    "N_chi=N_B=24^3": (2.0, 1e-26, 0, 200.0, 1e6, 1e4, 1e10, 1e10, 24 ** 3, 24 ** 3),
    "m_chi=10GeV": (10.0 / GEV_PER_MP, 1e-26, 0, 200.0, 5e6, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "m_chi=100MeV": (0.1 / GEV_PER_MP, 2e-27, 0, 200.0, 5e4, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "m_chi=10MeV": (0.01 / GEV_PER_MP, 2e-27, 0, 200.0, 5e3, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "sigma~v^-2": (2.0, 2e-33, -2, 200.0, 1e6, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "sigma~v^-4": (2.0, 5e-40, -4, 200.0, 1e6, 1e4, 1e10, 1e10, 32 ** 3, 32 ** 3),
    "F25 S3.4": (1.0, 1.6726e-23, 0, 0.0, 484.6, 72.69, 1e7, 1e7, 10 ** 5, 21 ** 3),
}


def setup(name, L=1.0, mu=1.0, seed=W.SEED_BASE + 900):
    """Initial conditions of a row: uniform positions, a Maxwellian dark matter with the row's
    bulk velocity along x and temperature, gas at rest at T_B0."""
    m_chi, s0, n, V0, Tc, Tb, rho_c, rho_b, Nc, Nb = ROWS[name]
    disp = float(np.sqrt(KB_OVER_MP * Tc / m_chi))
    w = W.box_workload(n_dm=Nc, n_gas=Nb, L=L, rho_dm=rho_c, rho_gas=rho_b, T_gas=Tb, sigma1d_dm=disp,
                       bulk_dm=(V0, 0.0, 0.0), m_chi_mp=m_chi, sigma0_cm2=s0, n=n,
                       v0_kms=C_KMS if n != 0 else 100.0, seed=seed, mu=mu)
    w["row"] = dict(name=name, m_chi=m_chi, sigma0_cm2=s0, n=n, V_chi0=V0, T_chi0=Tc, T_B0=Tb,
                    rho_chi=rho_c, rho_B=rho_b, N_chi=Nc, N_B=Nb, L=L, mu=mu)
    return w


def _moments(x):
    """Jarque-Bera statistic of each column of x (device tensor), without the factor N."""
    d = x - x.mean(0, keepdim=True)
    m2 = (d * d).mean(0)
    S = (d ** 3).mean(0) / m2 ** 1.5
    K = (d ** 4).mean(0) / (m2 * m2)
    return ((S * S + 0.25 * (K - 3.0) ** 2) / 6.0)


def diagnostics(dm, gas, m_chi):
    """Snapshot quantities of the device state (see the module docstring)."""
    import torch
    v, M = dm["vel"], dm["mass"]
    Vg, Mg, T, mu = gas["vel"], gas["mass"], gas["T"], gas["mu"]
    Mt, Mgt = M.sum(), Mg.sum()
    Vc = (M[:, None] * v).sum(0) / Mt
    th_c = ((M[:, None] * (v - Vc) ** 2).sum() / (3.0 * Mt))
    Vb = (Mg[:, None] * Vg).sum(0) / Mgt
    th_int = (Mg * KB_OVER_MP * T / mu).sum() / Mgt
    th_disp = (Mg[:, None] * (Vg - Vb) ** 2).sum() / (3.0 * Mgt)
    P = (M * v[:, 0]).sum() + (Mg * Vg[:, 0]).sum()
    E = (0.5 * M * (v * v).sum(1)).sum() + (Mg * (0.5 * (Vg * Vg).sum(1) + 1.5 * KB_OVER_MP * T / mu)).sum()
    jb = _moments(v)
    out = torch.stack([Vc[0], Vb[0], th_c, th_int + th_disp, th_int, th_disp, P, E, jb[0], jb[1], jb[2]])
    o = out.double().cpu().numpy()
    return dict(V_chi=o[0], V_B=o[1], theta_chi=o[2], theta_B=o[3], theta_B_internal=o[4],
                theta_B_dispersion=o[5], P=o[6], E=o[7], JB=o[8:11], rho_chi=float(Mt) / 1.0, rho_B=float(Mgt))


def run(name, t_end=1.0, dt=1e-3, snap=50, rate_mode=dmb.DMB_RATE_CLOSED, L=1.0, mu=1.0, seed=W.SEED_BASE + 900,
        rng_seed=7, beta=0.0):
    """Step a row from t = 0 to t_end; returns the snapshot series and the timing.  beta != 0
    makes the scattering anisotropic, dsigma/dOmega ~ 1 + beta cos theta (dmb_set_anisotropy)."""
    import torch
    w = setup(name, L, mu, seed)
    prm = w["params"]
    stream = torch.cuda.current_stream()
    ctx = dmb.Context(prm["sigma0_cm2"], prm["n"], prm["m_chi_mp"], prm["v0_kms"], True, tuple(prm["box"]), rng_seed,
                      rate_mode=rate_mode, stream=stream)
    if rate_mode == dmb.DMB_RATE_MLP:
        ctx.dmb_train_surrogate(nsamples=1 << 20, epochs=24, seed=11)
    if beta != 0.0:
        ctx.dmb_set_anisotropy(beta)
    dm, gas = dmb.to_device(w["dm"]), dmb.to_device(w["gas"])
    nsteps = int(round(t_end / dt))
    snaps, times, scat = [], [], 0
    # running totals of the step's sums: realised dark-matter kinetic-energy change, gas energy
    # change, expected dark-matter energy change, scatters, expected scatters (sum of P)
    budget = np.zeros(5)
    m_chi = w["row"]["m_chi"]
    snaps.append(diagnostics(dm, gas, m_chi))
    times.append(0.0)
    torch.cuda.synchronize()
    gpu_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    for k in range(nsteps):
        e0.record(stream)
        s = ctx.dmb_step(dm, gas, k, dt, want_sums=True)
        # drift, wrapped into the box
        dm["pos"].add_(dm["vel"], alpha=dt).remainder_(L)
        gas["pos"].add_(gas["vel"], alpha=dt).remainder_(L)
        e1.record(stream)
        e1.synchronize()
        gpu_ms += e0.elapsed_time(e1)
        scat += int(s[9])
        budget += s[[6, 7, 8, 9, 13]]
        if (k + 1) % snap == 0 or k + 1 == nsteps:
            snaps.append(diagnostics(dm, gas, m_chi))
            times.append((k + 1) * dt)
    wall = time.perf_counter() - t0
    keys = [k for k in snaps[0] if k not in ("rho_chi", "rho_B")]
    series = {k: np.array([sn[k] for sn in snaps]) for k in keys}
    series["t"] = np.array(times)
    budget = dict(dE_chi=budget[0], dE_gas=budget[1], dE_chi_expected=budget[2], scatters=budget[3],
                  scatters_expected=budget[4])
    return dict(row=dict(w["row"], beta=beta), series=series, steps=nsteps, dt=dt, scatters=scat, budget=budget,
                ms_per_step=gpu_ms / nsteps,
                wall_s=wall, n_pairs=int(s[12]), rho=(snaps[0]["rho_chi"] / L ** 3, snaps[0]["rho_B"] / L ** 3))
