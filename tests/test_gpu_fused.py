"""The fused pair pass of a float32 step (dmb_set_fusion(ctx, 1)): one sweep over the
gas-major pairs evaluates each pair's geometry and overlap once for the mean field (Eqs.
gas-dVdt, gas-dTdt) and for P_ij (Eq. dm-update-prob); the Monte Carlo then sums and selects per
DM row from those probabilities.  It must give the separate passes' results bit for bit: the
same arithmetic on the same pairs, exact fixed-point probability sums.  (The separate passes are
checked against the oracle in tests/test_gpu_parity.py and the others.)"""
import numpy as np
import pytest

from gpu_common import require_gpu, torch
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _ctx(w, fuse, rate=dmb.DMB_RATE_CLOSED, beta=0.0, screened=None):
    p = w["params"]
    c = dmb.Context(p["sigma0_cm2"], p["n"], p["m_chi_mp"], p["v0_kms"], p["periodic"], tuple(p["box"]), p["seed"],
                    rate_mode=rate)
    c.dmb_set_fusion(fuse)
    if beta:
        c.dmb_set_anisotropy(beta)
    if screened:
        c.dmb_set_cross_section(1, screened)
    return c


def _steps(c, w, nsteps, dt, batched=False):
    dm, gas = dmb.to_device(w["dm"]), dmb.to_device(w["gas"])
    out = []
    for s in range(nsteps):
        if batched:
            db = torch.from_numpy(w["dm_box"].view(np.int32)).cuda()
            gb = torch.from_numpy(w["gas_box"].view(np.int32)).cuda()
            sums = c.dmb_step_batched(dm, db, gas, gb, w["boxes"], s, dt)
        else:
            sums = c.dmb_step(dm, gas, s, dt)
        torch.cuda.synchronize()
        out.append((sums, dm["vel"].cpu().numpy(), gas["vel"].cpu().numpy(), gas["T"].cpu().numpy()))
    return out


def _same(a, b):
    for (sa, va, Va, Ta), (sb, vb, Vb, Tb) in zip(a, b):
        assert np.array_equal(sa, sb), sa - sb
        assert np.array_equal(va, vb) and np.array_equal(Va, Vb) and np.array_equal(Ta, Tb)


@pytest.mark.parametrize("name", ["box4k", "galaxy1M"])
def test_fused_step_equals_separate_passes(name):
    w = W.named(name, n=-2) if name == "galaxy1M" else W.named(name)
    dt = w["dt"] * (30.0 if name == "box4k" else 2000.0)  # enough scatters to exercise the selection
    a = _steps(_ctx(w, True), w, 3, dt)
    b = _steps(_ctx(w, False), w, 3, dt)
    assert a[-1][0][9] > 50                                # scatters
    _same(a, b)


def test_fused_step_with_other_providers_and_laws():
    w = W.box_workload(n_dm=3000, n_gas=2500, seed=71, n=-2)
    for kw in (dict(rate=dmb.DMB_RATE_QUAD), dict(beta=0.7), dict(rate=dmb.DMB_RATE_QUAD, screened=60.0)):
        a = _steps(_ctx(w, True, **kw), w, 2, w["dt"] * 50.0)
        b = _steps(_ctx(w, False, **kw), w, 2, w["dt"] * 50.0)
        _same(a, b)
    # the learned surrogate (the same network in both contexts); the fused pass reads stored
    # rates, so the separate passes must store them too (mode 1 of dmb_set_surrogate_epilogue sums
    # the mean field inside the surrogate's kernel, in another float32 order)
    ca, cb = _ctx(w, True, rate=dmb.DMB_RATE_MLP), _ctx(w, False, rate=dmb.DMB_RATE_MLP)
    cb.dmb_set_surrogate_epilogue(0)
    ca.dmb_train_surrogate(nsamples=1 << 15, epochs=2, seed=4)
    cb.dmb_load_surrogate(ca.dmb_surrogate_params())
    _same(_steps(ca, w, 2, w["dt"] * 50.0), _steps(cb, w, 2, w["dt"] * 50.0))


def test_fused_batched_step_with_and_without_graph():
    w = W.boxes_workload(nbox=5, n_lo=800, n_hi=4000, seed=72, dt=2e-3)
    ref = _steps(_ctx(w, False), w, 3, w["dt"], batched=True)
    _same(_steps(_ctx(w, True), w, 3, w["dt"], batched=True), ref)
    g = _ctx(w, True)
    g.dmb_set_graph(True)
    _same(_steps(g, w, 3, w["dt"], batched=True), ref)
