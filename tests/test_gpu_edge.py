"""Edge cases of the CUDA path through the C ABI."""
import numpy as np
import pytest

from gpu_common import device_inputs, gpu_pairs, make_ctx, require_gpu, torch
from oracle.pairs import pairs_bruteforce
from oracle.step import oracle_step
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def _box(nd, ng, **kw):
    """A periodic box with nd DM and ng gas (either may be 0); h capped at L/8 so the
    minimum image stays unambiguous for small particle numbers."""
    w = W.box_workload(n_dm=max(nd, 1), n_gas=max(ng, 1), seed=123 + nd + 7 * ng, **kw)
    L = w["params"]["box"][0]
    for sp, n in (("dm", nd), ("gas", ng)):
        w[sp] = {k: v[:n].copy() for k, v in w[sp].items()}
        w[sp]["h"] = np.minimum(w[sp]["h"], L / 8)
    return w


@pytest.mark.parametrize("nd,ng", [(0, 50), (50, 0), (1, 1), (33, 65), (31, 1000), (1025, 33)])
def test_ragged_and_empty(nd, ng):
    w = _box(nd, ng)
    if nd * ng > 0 and nd * ng < 2000:
        # make sure some pairs exist for tiny inputs
        w["dm"]["h"][:] = 0.12
        w["gas"]["h"][:] = 0.12
        w["gas"]["pos"][0] = w["dm"]["pos"][0] + 0.01
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    gi, gj = gpu_pairs(ctx, dm, gas)
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    assert sorted(zip(gi.tolist(), gj.tolist())) == sorted(zip(pi.tolist(), pj.tolist()))
    sums = ctx.dmb_step(dm, gas, 1, w["dt"])
    ref = oracle_step(w["dm"], w["gas"], w["params"], 1, w["dt"])["sums"]
    assert sums[12] == ref[12] and sums[9] == ref[9]


def test_power_law_n_minus4_renormalises():
    # sigma ~ v^-4: slow relative speeds give P > 1; the draw is renormalised and counted
    w = _box(300, 300, n=-4, sigma0_cm2=1e-23, dt=5e-2)
    out = oracle_step(w["dm"], w["gas"], w["params"], 2, w["dt"])
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    sums = ctx.dmb_step(dm, gas, 2, w["dt"])
    assert out["sums"][10] > 0
    assert sums[10] == out["sums"][10]
    assert abs(sums[9] - out["sums"][9]) <= sums[15] + 0


def test_cold_gas():
    w = _box(400, 400, bulk_dm=(120.0, 0, 0))
    w["gas"]["T"][:] = 0.0
    out = oracle_step(w["dm"], w["gas"], w["params"], 4, w["dt"])
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    sums = ctx.dmb_step(dm, gas, 4, w["dt"])
    for k in (3, 4, 5, 8):
        assert abs(sums[k] - out["sums"][k]) <= 1e-4 * abs(out["sums"][k]) + 1e-12


def test_bad_inputs_are_rejected():
    w = _box(64, 64)
    w["gas"]["h"][3] = -1.0
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    with pytest.raises(dmb.DmbError) as e:
        ctx.dmb_neighbors()
    assert e.value.status == dmb.DMB_ERR_ARG
    w2 = _box(64, 64)
    w2["dm"]["pos"][0, 0] = np.nan
    ctx2 = make_ctx(w2)
    dm2, gas2 = device_inputs(w2)
    with pytest.raises(dmb.DmbError):
        ctx2.dmb_step(dm2, gas2, 0, w2["dt"])


def test_periodic_box_too_small():
    w = _box(64, 64)
    w["dm"]["h"][:] = 0.3
    w["gas"]["h"][:] = 0.3     # h_i + h_j = 0.6 > L/2
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    with pytest.raises(dmb.DmbError):
        ctx.dmb_neighbors()


def test_call_order_and_parameters():
    w = _box(16, 16)
    ctx = make_ctx(w)
    acc = torch.empty((16, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(dmb.DmbError) as e:
        ctx.dmb_meanfield_gas(acc, dudt)
    assert e.value.status == dmb.DMB_ERR_STATE
    with pytest.raises(dmb.DmbError) as e:
        dmb.Context(1e-24, -5, 2.0)
    assert e.value.status == dmb.DMB_ERR_ARG
    with pytest.raises(dmb.DmbError):
        dmb.Context(1e-24, 0, 2.0, rate_mode=7)
    with pytest.raises(dmb.DmbError):
        dmb.Context(1e-24, 0, 2.0, rate_mode=dmb.DMB_RATE_MLP, fp64=True)


def test_deterministic_repeat():
    w = _box(800, 800, bulk_dm=(100.0, 0, 0), dt=2e-3)
    outs = []
    for _ in range(2):
        ctx = make_ctx(w)
        dm, gas = device_inputs(w)
        outs.append((ctx.dmb_step(dm, gas, 9, w["dt"]), dm["vel"].cpu().numpy(), gas["T"].cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


def test_multi_step_matches_oracle_chain():
    # three consecutive steps through dmb_step against three oracle steps (float64 mode)
    w = _box(300, 300, bulk_dm=(150.0, 0, 0), dt=1e-3)
    ctx = make_ctx(w, fp64=True)
    dm, gas = device_inputs(w)
    dmo = {k: v.copy() for k, v in w["dm"].items()}
    gaso = {k: v.copy() for k, v in w["gas"].items()}
    for step in range(3):
        ctx.dmb_step(dm, gas, step, w["dt"])
        out = oracle_step(dmo, gaso, w["params"], step, w["dt"])
        dmo["vel"] = out["mc"]["vel_new"]
        gaso["vel"] = out["V_new"]
        gaso["T"] = out["T_new"]
    np.testing.assert_allclose(dm["vel"].cpu().numpy(), dmo["vel"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gas["T"].cpu().numpy(), gaso["T"], rtol=1e-10)
