"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws particles: positions, velocities, masses, smoothing
lengths, temperatures and ids.  It holds none of the interaction method's
arithmetic (no overlap integral, no rates, no probabilities), so both the CUDA
path and the oracle read their inputs from it.

Units: kpc, km/s, Msun, K; particle masses m_chi, mu in m_p.

Workloads
  box4k      periodic 1 kpc box, 4096 DM + 4096 gas, uniform positions, gas at rest
             at T = 1e4 K, DM Maxwellian with 1D dispersion 100 km/s, equal particle
             masses for rho_chi = rho_B = 1e10 Msun/kpc^3 (the paper's standard
             densities, App. F), m_chi = 2 m_p, sigma = 1e-24 cm^2, n = 0,
             h for 32 same-species neighbours: h = (3*32 / (4 pi n))^(1/3).
  galaxy     Hernquist halo (a = 20 kpc, M = 1e12 Msun, truncated at 10a) of DM with
             isotropic Jeans velocities + exponential gas disk (R_d = 3 kpc,
             z_d = 0.3 kpc, M_gas = 0.2 x 4.297e10 Msun, the paper's AGORA gas
             fraction), rotating with the circular velocity of the enclosed mass,
             T = 1e4 K; h from the analytic local density for 32 neighbours, floored
             at the paper's 44.8 pc (Sec. 4).
  boxes      many independent periodic boxes of uneven size and parameters.
  galaxy40M  the galaxy geometry at 32M DM + 8M gas, sigma = 3e-26 cm^2, with seeded
             power-of-two timestep bins (timestep_bins) for hierarchical substeps.
"""
import math

import numpy as np

G_KPC = 4.30091e-6          # gravitational constant [kpc (km/s)^2 / Msun]
NGB = 32                    # neighbours the smoothing length is set for
H_FLOOR_KPC = 0.0448        # interaction-softening floor of the paper's galaxy runs
SEED_BASE = 0x260324688


def _h_from_number_density(n):
    return (3.0 * NGB / (4.0 * math.pi * n)) ** (1.0 / 3.0)


def _particles(pos, vel, mass, h, ids):
    return dict(pos=np.ascontiguousarray(pos, dtype=np.float64),
                vel=np.ascontiguousarray(vel, dtype=np.float64),
                mass=np.ascontiguousarray(mass, dtype=np.float64),
                h=np.ascontiguousarray(h, dtype=np.float64),
                id=np.ascontiguousarray(ids, dtype=np.uint32))


def _params(sigma0_cm2, n, m_chi_mp, periodic, box, seed, v0_kms=100.0):
    return dict(sigma0_cm2=float(sigma0_cm2), v0_kms=float(v0_kms), n=int(n),
                m_chi_mp=float(m_chi_mp), periodic=bool(periodic),
                box=np.asarray(box, dtype=np.float64), seed=int(seed))


def box_workload(n_dm=4096, n_gas=4096, L=1.0, rho=1e10, T_gas=1e4, sigma1d_dm=100.0,
                 bulk_dm=(0.0, 0.0, 0.0), m_chi_mp=2.0, sigma0_cm2=1e-24, n=0, v0_kms=100.0,
                 dt=1e-4, seed=SEED_BASE + 1, rho_dm=None, rho_gas=None, mu=1.0):
    """Uniform periodic box (the App. F test-problem geometry at a chosen size)."""
    rng = np.random.default_rng(seed)
    rho_dm = rho if rho_dm is None else rho_dm
    rho_gas = rho if rho_gas is None else rho_gas
    vol = L ** 3
    dm = _particles(rng.uniform(0.0, L, (n_dm, 3)),
                    np.asarray(bulk_dm)[None, :] + sigma1d_dm * rng.standard_normal((n_dm, 3)),
                    np.full(n_dm, rho_dm * vol / n_dm),
                    np.full(n_dm, _h_from_number_density(n_dm / vol)),
                    np.arange(n_dm))
    gas = _particles(rng.uniform(0.0, L, (n_gas, 3)), np.zeros((n_gas, 3)),
                     np.full(n_gas, rho_gas * vol / n_gas),
                     np.full(n_gas, _h_from_number_density(n_gas / vol)),
                     np.arange(n_gas))
    gas["T"] = np.full(n_gas, float(T_gas))
    gas["mu"] = np.full(n_gas, float(mu))
    params = _params(sigma0_cm2, n, m_chi_mp, True, (L, L, L), seed, v0_kms)
    return dict(name=f"box{n_dm}+{n_gas}", dm=dm, gas=gas, params=params, dt=float(dt))


# ---- galaxy ----------------------------------------------------------------------

def _hernquist_mass(r, M, a):
    return M * r * r / (r + a) ** 2


def _hernquist_rho(r, M, a):
    return M * a / (2.0 * math.pi * r * (r + a) ** 3)


def _hernquist_sigma_r(r, M, a, rmax):
    """Isotropic Jeans dispersion sigma_r(r) of a Hernquist sphere (numerical)."""
    grid = np.geomspace(1e-4 * a, 1e4 * a, 20000)
    rho = _hernquist_rho(grid, M, a)
    integrand = rho * G_KPC * _hernquist_mass(grid, M, a) / grid ** 2
    # cumulative integral from r to the outer edge of the grid
    seg = 0.5 * (integrand[1:] + integrand[:-1]) * np.diff(grid)
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    s2 = tail / rho
    return np.sqrt(np.interp(r, grid, s2))


def galaxy_workload(n_dm=1_000_000, n_gas=1_000_000, M_halo=1e12, a=20.0, R_d=3.0, z_d=0.3,
                    M_gas=0.2 * 4.297e10, T_gas=1e4, m_chi_mp=2.0, sigma0_cm2=1e-24, n=0,
                    v0_kms=100.0, dt=1e-4, seed=SEED_BASE + 2, mu=1.0):
    """Hernquist DM halo + exponential gas disk, centred on the origin."""
    rng = np.random.default_rng(seed)
    rmax = 10.0 * a
    M_trunc = _hernquist_mass(rmax, M_halo, a)
    # DM radii: invert M(<r)/M_trunc = u  ->  r = a sqrt(y) / (1 - sqrt(y)), y = u M_trunc / M
    y = rng.uniform(0.0, 1.0, n_dm) * (M_trunc / M_halo)
    sy = np.sqrt(y)
    r = a * sy / (1.0 - sy)
    cth = rng.uniform(-1.0, 1.0, n_dm)
    ph = rng.uniform(0.0, 2.0 * math.pi, n_dm)
    sth = np.sqrt(1.0 - cth * cth)
    dm_pos = np.stack([r * sth * np.cos(ph), r * sth * np.sin(ph), r * cth], axis=1)
    sig = _hernquist_sigma_r(r, M_halo, a, rmax)
    dm_vel = sig[:, None] * rng.standard_normal((n_dm, 3))
    m_dm = M_trunc / n_dm
    n_dm_density = _hernquist_rho(np.maximum(r, 1e-6), M_halo, a) / m_dm
    h_dm = np.maximum(_h_from_number_density(n_dm_density), H_FLOOR_KPC)

    # gas disk: R ~ R_d * Gamma(2), |z| ~ Exp(z_d), truncated at 10 R_d and 10 z_d
    R = rng.gamma(2.0, R_d, n_gas)
    while np.any(R > 10.0 * R_d):
        bad = R > 10.0 * R_d
        R[bad] = rng.gamma(2.0, R_d, int(bad.sum()))
    z = rng.exponential(z_d, n_gas)
    while np.any(z > 10.0 * z_d):
        bad = z > 10.0 * z_d
        z[bad] = rng.exponential(z_d, int(bad.sum()))
    z *= rng.choice([-1.0, 1.0], n_gas)
    phg = rng.uniform(0.0, 2.0 * math.pi, n_gas)
    gas_pos = np.stack([R * np.cos(phg), R * np.sin(phg), z], axis=1)
    # circular speed from the enclosed (spherical) halo + disk mass
    M_disk_enc = M_gas * (1.0 - np.exp(-R / R_d) * (1.0 + R / R_d))
    vc = np.sqrt(G_KPC * (_hernquist_mass(R, M_halo, a) + M_disk_enc) / R)
    gas_vel = np.stack([-vc * np.sin(phg), vc * np.cos(phg), np.zeros(n_gas)], axis=1)
    m_gas = M_gas / n_gas
    rho_gas = M_gas / (4.0 * math.pi * R_d ** 2 * z_d) * np.exp(-R / R_d) * np.exp(-np.abs(z) / z_d)
    h_gas = np.maximum(_h_from_number_density(rho_gas / m_gas), H_FLOOR_KPC)

    dm = _particles(dm_pos, dm_vel, np.full(n_dm, m_dm), h_dm, np.arange(n_dm))
    gas = _particles(gas_pos, gas_vel, np.full(n_gas, m_gas), h_gas, np.arange(n_gas))
    gas["T"] = np.full(n_gas, float(T_gas))
    gas["mu"] = np.full(n_gas, float(mu))
    params = _params(sigma0_cm2, n, m_chi_mp, False, (0.0, 0.0, 0.0), seed, v0_kms)
    return dict(name=f"galaxy{n_dm}+{n_gas}", dm=dm, gas=gas, params=params, dt=float(dt))


def boxes_workload(nbox=64, n_lo=2 ** 12, n_hi=2 ** 18, sigma_lo=1e-27, sigma_hi=1e-24, m_lo=0.5, m_hi=10.0,
                   T_lo=1e3, T_hi=1e6, L=1.0, rho=1e10, sigma1d_dm=100.0, n=0, v0_kms=100.0, dt=1e-4,
                   seed=SEED_BASE + 4):
    """Many independent periodic boxes: particle counts per species, sigma0, m_chi and the gas
    temperature drawn log-uniformly per box (a parameter scan over boxes).  Returns the boxes'
    particles concatenated (with per-particle box indices), the per-box parameters and each
    box's own workload dict."""
    rng = np.random.default_rng(seed)
    lu = lambda a, b: float(np.exp(rng.uniform(np.log(a), np.log(b))))
    per = []
    for b in range(nbox):
        nd = int(round(lu(n_lo, n_hi)))
        ng = int(round(lu(n_lo, n_hi)))
        w = box_workload(n_dm=nd, n_gas=ng, L=L, rho=rho, T_gas=lu(T_lo, T_hi), sigma1d_dm=sigma1d_dm,
                         m_chi_mp=lu(m_lo, m_hi), sigma0_cm2=lu(sigma_lo, sigma_hi), n=n, v0_kms=v0_kms, dt=dt,
                         seed=seed * 1000 + b)
        per.append(w)
    cat = lambda sp, k: np.concatenate([w[sp][k] for w in per])
    dm = {k: cat("dm", k) for k in per[0]["dm"]}
    gas = {k: cat("gas", k) for k in per[0]["gas"]}
    # ids unique across boxes (the Philox streams key on ids)
    dm["id"] = np.arange(len(dm["h"]), dtype=np.uint32)
    gas["id"] = np.arange(len(gas["h"]), dtype=np.uint32)
    dm_box = np.concatenate([np.full(len(w["dm"]["h"]), b, np.uint32) for b, w in enumerate(per)])
    gas_box = np.concatenate([np.full(len(w["gas"]["h"]), b, np.uint32) for b, w in enumerate(per)])
    boxes = [(tuple(w["params"]["box"]), w["params"]["sigma0_cm2"], w["params"]["m_chi_mp"]) for w in per]
    params = _params(1e-24, n, 2.0, True, (L, L, L), seed, v0_kms)
    return dict(name=f"boxes{nbox}", dm=dm, gas=gas, dm_box=dm_box, gas_box=gas_box, boxes=boxes, per_box=per,
                params=params, dt=float(dt))


def timestep_bins(n, seed, f_lo=0.01, f_hi=0.1, top=10):
    """Seeded power-of-two timestep bins (uint8): P(bin <= v) = f_lo (f_hi / f_lo)^(v / top) for
    v = 0 .. top, the rest in bin top + 1.  A particle in bin b is active at substep s when
    s mod 2^b == 0, so every substep 0 < s < 2^(top+1) has between f_lo and f_hi of the
    particles active."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, n)
    F = f_lo * (f_hi / f_lo) ** (np.arange(top + 1) / top)
    return np.searchsorted(F, u, side="right").astype(np.uint8)


def subsample(w, frac_or_n_dm, n_gas=None, seed=0):
    """A smaller workload with the same structure (random particle subsets)."""
    rng = np.random.default_rng(seed)
    nd = len(w["dm"]["h"])
    ng = len(w["gas"]["h"])
    kd = frac_or_n_dm if n_gas is not None else int(nd * frac_or_n_dm)
    kg = n_gas if n_gas is not None else int(ng * frac_or_n_dm)
    sd = np.sort(rng.choice(nd, kd, replace=False))
    sg = np.sort(rng.choice(ng, kg, replace=False))
    out = dict(w)
    out["dm"] = {k: v[sd] for k, v in w["dm"].items()}
    out["gas"] = {k: v[sg] for k, v in w["gas"].items()}
    return out


def named(name, **kw):
    """Workloads by name: 'box4k', 'box4k-bulk', 'galaxy1M', 'galaxy10M', 'galaxy40M'."""
    if name == "box4k":
        return box_workload(**kw)
    if name == "box4k-bulk":
        return box_workload(bulk_dm=(200.0, 0.0, 0.0), **kw)
    if name == "galaxy1M":
        return galaxy_workload(1_000_000, 1_000_000, seed=SEED_BASE + 2, **kw)
    if name == "galaxy40M":
        kw.setdefault("sigma0_cm2", 3e-26)
        w = galaxy_workload(32_000_000, 8_000_000, seed=SEED_BASE + 5, **kw)
        w["dm_bin"] = timestep_bins(32_000_000, SEED_BASE + 51)
        w["gas_bin"] = timestep_bins(8_000_000, SEED_BASE + 52)
        return w
    if name == "galaxy10M":
        return galaxy_workload(8_000_000, 2_000_000, seed=SEED_BASE + 3, **kw)
    raise KeyError(name)
