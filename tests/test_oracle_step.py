"""Pins for the oracle's mean field and step: App. C identities and the step's sums."""
import numpy as np

from oracle import units
from oracle.expect import expected_dm, pair_budget
from oracle.meanfield import meanfield_gas
from oracle.pairs import pairs_bruteforce
from oracle.step import oracle_step
from paper_2603_24688_gb300 import workloads as W


def _w(n=0, **kw):
    return W.box_workload(n_dm=256, n_gas=256, seed=9, n=n, bulk_dm=(150.0, -20.0, 0.0), **kw)


def test_pairwise_conservation_in_expectation():
    # App. C: M_i E[dv_i] + M_j dV_j/dt dt = 0 and the energy identity, pair by pair
    for n in (-4, -2, 0, 2):
        w = _w(n)
        pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
        dp, dE, sp, sE = pair_budget(w["dm"], w["gas"], pi, pj, w["params"], w["dt"])
        assert np.all(np.abs(dp) <= 1e-12 * sp[:, None])
        assert np.all(np.abs(dE) <= 1e-12 * sE)


def test_gas_transfer_equals_minus_expected_dm_transfer():
    w = _w(0)
    dm, gas, prm, dt = w["dm"], w["gas"], w["params"], w["dt"]
    pi, pj = pairs_bruteforce(dm, gas, True, prm["box"])
    acc, dudt = meanfield_gas(dm, gas, pi, pj, prm)
    E_dv, E_dE, _ = expected_dm(dm, gas, pi, pj, prm, dt)
    p_gas = (gas["mass"][:, None] * acc * dt).sum(0)
    p_dm = (dm["mass"][:, None] * E_dv).sum(0)
    assert np.allclose(p_gas, -p_dm, rtol=1e-12, atol=1e-12 * np.abs(p_gas).max())
    e_gas = (gas["mass"] * (dudt + np.sum(gas["vel"] * acc, 1)) * dt).sum()
    assert abs(e_gas + E_dE.sum()) < 1e-11 * abs(E_dE).sum()


def test_heating_sign_hot_dm_heats_cold_gas():
    # DM far hotter than the gas: the gas heats (du/dt > 0 on average) and is dragged along
    # the DM bulk flow (mean acceleration along +x)
    w = _w(0)
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    acc, dudt = meanfield_gas(w["dm"], w["gas"], pi, pj, w["params"])
    assert dudt.mean() > 0
    assert acc[:, 0].mean() > 0


def test_step_sums_and_kicks():
    w = _w(0)
    out = oracle_step(w["dm"], w["gas"], w["params"], 3, w["dt"])
    s = out["sums"]
    dt = w["dt"]
    gas = w["gas"]
    assert np.allclose(s[3:6], (gas["mass"][:, None] * out["acc"] * dt).sum(0))
    assert np.allclose(out["V_new"], gas["vel"] + out["acc"] * dt)
    u0 = units.u_from_T(gas["T"], gas["mu"])
    np.testing.assert_allclose(units.u_from_T(out["T_new"], gas["mu"]), u0 + out["dudt"] * dt, rtol=1e-12)
    # first-order energy budget: gas energy gain = - expected DM energy change, up to the
    # second-order kinetic term (1/2) M |a dt|^2
    second = (0.5 * gas["mass"] * np.sum((out["acc"] * dt) ** 2, 1)).sum()
    assert abs(s[7] + s[8] - second) < 1e-9 * abs(s[8])
    assert s[9] == out["mc"]["scattered"].sum()
    assert s[12] == len(out["pairs"][0])


def test_thermal_energy_clamp():
    # a gas particle that would go below u = 0 is clamped and counted
    w = _w(0, T_gas=1.0)
    w["dm"]["vel"][:] = w["gas"]["vel"][0]     # DM at rest relative to the gas: pure cooling
    w["gas"]["T"][:] = 1e6
    w["dt"] = 50.0
    out = oracle_step(w["dm"], w["gas"], w["params"], 0, w["dt"])
    assert out["sums"][11] > 0
    assert np.all(out["u_new"] >= 0)
