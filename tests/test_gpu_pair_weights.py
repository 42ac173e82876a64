"""Pair weights of a float32 pair set (dmb_set_pair_weights): the search's emit pass forms each
pair's overlap g_ij (Eqs. gas-dVdt, dm-update-prob) with the same canonical displacement and
overlap-table arithmetic as the interaction kernels, and stores M_i g_ij and g_ij beside the
pair lists; the mean field and the Monte Carlo read them.  Whichever way g_ij is formed, the
results must be the same bit for bit (the oracle parity of the default path is checked in
tests/test_gpu_parity.py and the others)."""
import numpy as np
import pytest

from gpu_common import device_inputs, require_gpu, torch
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _ctx(w, mode, rate=dmb.DMB_RATE_CLOSED):
    p = w["params"]
    c = dmb.Context(p["sigma0_cm2"], p["n"], p["m_chi_mp"], p["v0_kms"], p["periodic"], tuple(p["box"]), p["seed"],
                    rate_mode=rate)
    c.dmb_set_pair_weights(mode)
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
def test_steps_with_stored_weights_equal_the_default(name):
    w = W.named(name, n=-2) if name == "galaxy1M" else W.named(name)
    dt = w["dt"] * (30.0 if name == "box4k" else 2000.0)   # enough scatters to exercise the selection
    a = _steps(_ctx(w, 1), w, 3, dt)
    b = _steps(_ctx(w, -1), w, 3, dt)
    assert a[-1][0][9] > 50                                # scatters
    _same(a, b)


def test_batched_steps_with_stored_weights_and_graphs():
    w = W.boxes_workload(nbox=5, n_lo=800, n_hi=4000, seed=74, dt=2e-3)
    ref = _steps(_ctx(w, 0), w, 3, w["dt"], batched=True)
    _same(_steps(_ctx(w, 1), w, 3, w["dt"], batched=True), ref)
    g = _ctx(w, 1)
    g.dmb_set_graph(True)
    _same(_steps(g, w, 3, w["dt"], batched=True), ref)


@pytest.mark.parametrize("rate", [dmb.DMB_RATE_CLOSED, dmb.DMB_RATE_QUAD])
def test_standalone_calls_on_a_kept_pair_set(rate):
    # dmb_neighbors keeps its pair set: by default it stores the weights, and the standalone mean
    # field and Monte Carlo read them; mode 0 forms g in the kernels
    w = W.subsample(W.named("galaxy1M", n=-2), 60_000, 40_000, seed=3)
    out = {}
    for mode in (-1, 0):
        c = _ctx(w, mode, rate)
        dm, gas = device_inputs(w)
        c.dmb_build_grid(dm, gas)
        n = c.dmb_neighbors()
        nb, nd = len(w["gas"]["h"]), len(w["dm"]["h"])
        acc = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
        dudt = torch.empty(nb, dtype=torch.float64, device="cuda")
        c.dmb_meanfield_gas(acc, dudt)
        vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
        sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
        pa = torch.empty(nd, dtype=torch.int32, device="cuda")
        pt = torch.empty(nd, dtype=torch.float64, device="cuda")
        c.dmb_mc_scatter_dm(5, 0.2, vel, sc, pa, None, pt)   # a long step: scatters to select
        torch.cuda.synchronize()
        out[mode] = [n] + [t.cpu().numpy() for t in (acc, dudt, vel, sc, pa, pt)]
    assert out[-1][0] == out[0][0] > 100_000
    for x, y in zip(out[-1][1:], out[0][1:]):
        assert np.array_equal(x, y)
    assert out[0][4].sum() > 0                         # some scatters


def test_substeps_with_and_without_weights():
    w = W.box_workload(n_dm=2000, n_gas=2100, seed=31, n=0, T_gas=3e4, bulk_dm=(150.0, 0.0, 0.0))
    rng = np.random.default_rng(2)
    db = rng.integers(0, 4, 2000).astype(np.uint8)
    gb = rng.integers(0, 4, 2100).astype(np.uint8)
    runs = []
    for mode, graph in ((-1, False), (0, False), (-1, True)):
        c = _ctx(w, mode)
        dm, gas = device_inputs(w)
        c.dmb_build_grid(dm, gas)
        c.dmb_neighbors()
        c.dmb_set_bins(torch.from_numpy(db).cuda(), torch.from_numpy(gb).cuda())
        c.dmb_set_graph(graph)
        res = []
        for s in (1, 2, 3, 4, 8, 1):
            res.append(c.dmb_substep(dm, gas, s, w["dt"]))
        torch.cuda.synchronize()
        runs.append((res, dm["vel"].cpu().numpy(), gas["vel"].cpu().numpy(), gas["T"].cpu().numpy()))
    for r in runs[1:]:
        for sa, sb in zip(runs[0][0], r[0]):
            assert np.array_equal(sa, sb)
        for x, y in zip(runs[0][1:], r[1:]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("kw", [dict(beta=0.6), dict(rate=dmb.DMB_RATE_QUAD, screened=60.0)])
def test_steps_with_weights_under_other_laws(kw):
    # anisotropic angles and the screened velocity law act on the pair's probability and kick,
    # not on g_ij: the stored weights serve them unchanged
    w = W.box_workload(n_dm=3000, n_gas=2500, seed=75, n=-2)
    runs = []
    for mode in (1, 0):
        c = _ctx(w, mode, kw.get("rate", dmb.DMB_RATE_CLOSED))
        if "beta" in kw:
            c.dmb_set_anisotropy(kw["beta"])
        if "screened" in kw:
            c.dmb_set_cross_section(1, kw["screened"])
        runs.append(_steps(c, w, 2, w["dt"] * 50.0))
    _same(runs[0], runs[1])


def test_mode_argument_checked():
    c = _ctx(W.named("box4k"), -1)
    with pytest.raises(dmb.DmbError):
        c.dmb_set_pair_weights(2)
    for m in (1, 0, -1):
        c.dmb_set_pair_weights(m)
