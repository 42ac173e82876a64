"""Config 2 over time: 100 steps of the 1M DM + 1M gas galaxy (sigma = 1e-24 cm^2, n = 0, float32
pair arithmetic with float64 per-gas sums), with oracle parity at steps 0, 1 and 99.

At each checked step the oracle restarts from the GPU's own state at that step (velocities and
temperatures after the earlier kicks and scatters) and evaluates sampled particles one by one:
the gas mean field (Eqs. gas-dVdt, gas-dTdt) and the Monte Carlo (Eqs. dm-update-vels,
dm-update-prob, scatter_chi, with the step index keying the Philox streams).  The step itself
(dmb_step) must reproduce the standalone calls: the DM velocities bit for bit, the gas kicks
V + a dt and u + (du/dt) dt to float64 rounding.
"""
import numpy as np
import pytest

from gpu_common import device_inputs, make_ctx, require_gpu, torch
from oracle import units
from oracle.mc import mc_scatter
from oracle.meanfield import meanfield_gas
from oracle.pairs import pairs_bruteforce
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CHECK = (0, 1, 99)


def _host_state(w, dm, gas):
    hs = {"dm": dict(w["dm"]), "gas": dict(w["gas"])}
    hs["dm"]["vel"] = dm["vel"].cpu().numpy().copy()
    hs["gas"]["vel"] = gas["vel"].cpu().numpy().copy()
    hs["gas"]["T"] = gas["T"].cpu().numpy().copy()
    return hs


def test_hundred_steps_with_parity_at_steps_0_1_99():
    require_gpu()
    w = W.named("galaxy1M")
    p, dt = w["params"], w["dt"]
    ctx = make_ctx(w)
    chk = make_ctx(w)                 # standalone calls on the current state
    dm, gas = device_inputs(w)
    nb, nd = len(w["gas"]["h"]), len(w["dm"]["h"])
    rng = np.random.default_rng(99)
    gs = rng.choice(nb, 24, replace=False)
    r = np.linalg.norm(w["dm"]["pos"], axis=1)
    near = np.nonzero((np.abs(w["dm"]["pos"][:, 2]) < 1.0) & (r < 12.0))[0]
    ds = rng.choice(near, 48, replace=False)
    # positions do not change in the interaction step, so the sampled rows' pairs are fixed
    gpi, gpj = pairs_bruteforce(w["dm"], w["gas"], False, None, gas_subset=gs, block=200000)
    dpi, dpj = pairs_bruteforce(w["dm"], w["gas"], False, None, dm_subset=ds, block=8)
    acc = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(nb, dtype=torch.float64, device="cuda")
    vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
    pa = torch.empty(nd, dtype=torch.int32, device="cuda")
    pt = torch.empty(nd, dtype=torch.float64, device="cuda")
    n_checked_scatters = 0
    for step in range(100):
        if step in CHECK:
            hs = _host_state(w, dm, gas)
            chk.dmb_build_grid(dm, gas)
            chk.dmb_neighbors()
            chk.dmb_meanfield_gas(acc, dudt)
            chk.dmb_mc_scatter_dm(step, dt, vel, sc, pa, None, pt)
            torch.cuda.synchronize()
            # gas mean field of the sampled rows against the oracle on this state
            a_ref, u_ref = meanfield_gas(hs["dm"], hs["gas"], gpi, gpj, p)
            a_got, u_got = acc.cpu().numpy(), dudt.cpu().numpy()
            err = np.linalg.norm(a_got[gs] - a_ref[gs], axis=1) / np.linalg.norm(a_ref[gs], axis=1)
            assert np.all(err < 1e-5), (step, err.max())
            scale = np.abs(u_ref[gs]) + 1e-3 * np.abs(u_ref[gs]).max()
            assert np.all(np.abs(u_got[gs] - u_ref[gs]) / scale < 1e-5), step
            # Monte Carlo of the sampled DM rows
            out = mc_scatter(hs["dm"], hs["gas"], dpi, dpj, p, step, dt)
            got_s = sc.cpu().numpy().astype(bool)[ds]
            got_p = pa.cpu().numpy().view(np.uint32).astype(np.uint64)[ds]
            np.testing.assert_allclose(pt.cpu().numpy()[ds], out["C_total"][ds], rtol=2e-5)
            band = out["gap"][ds] <= 1e-6
            mism = (got_s != out["scattered"][ds]) | (got_p != out["partner"][ds])
            assert not np.any(mism & ~band), step
            ok = out["scattered"][ds] & ~mism
            dv = vel.cpu().numpy()[ds][ok] - hs["dm"]["vel"][ds][ok]
            dv_ref = out["vel_new"][ds][ok] - hs["dm"]["vel"][ds][ok]
            assert np.all(np.linalg.norm(dv - dv_ref, axis=1) <= 1e-5 * np.linalg.norm(dv_ref, axis=1) + 1e-9)
            n_checked_scatters += int(ok.sum())
            vel_mc, a_all, u_all = vel.clone(), acc.clone(), dudt.clone()
        sums = ctx.dmb_step(dm, gas, step, dt)
        assert np.isfinite(sums).all()
        if step in CHECK:
            torch.cuda.synchronize()
            # the step's updates are the standalone results applied with dt
            assert torch.equal(dm["vel"], vel_mc), step
            v_exp = hs["gas"]["vel"] + a_all.cpu().numpy() * dt
            np.testing.assert_allclose(gas["vel"].cpu().numpy(), v_exp, rtol=1e-14, atol=1e-12)
            u0 = units.u_from_T(hs["gas"]["T"], hs["gas"]["mu"])
            u1 = np.maximum(u0 + u_all.cpu().numpy() * dt, 0.0)
            np.testing.assert_allclose(gas["T"].cpu().numpy(), units.T_from_u(u1, hs["gas"]["mu"]), rtol=1e-12)
    print("scatters checked against the oracle:", n_checked_scatters)
