"""GPU parity of hierarchical substeps (power-of-two timestep bins) against the oracle's
substep, and CUDA-graph replay against direct launches.

Tolerances as in the full-step parity tests: transfers within 1e-5 (float32 pairs) and 1e-12
(float64) relative, Monte Carlo decisions identical.
"""
import numpy as np
import pytest

from gpu_common import device_inputs, make_ctx, require_gpu, torch
from oracle.pairs import pairs_bruteforce
from oracle.substep import active_mask, oracle_substep
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _w():
    return W.box_workload(n_dm=2000, n_gas=2100, seed=31, n=0, T_gas=3e4, bulk_dm=(150.0, 0.0, 0.0))


def _bins(n, seed, top=3):
    return np.random.default_rng(seed).integers(0, top + 1, n).astype(np.uint8)


def _u8(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def _copy(p):
    return {k: v.copy() for k, v in p.items()}


def _setup(w, db, gb, fp64=False, graph=False):
    ctx = make_ctx(w, fp64=fp64)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    dbd, gbd = _u8(db), _u8(gb)
    ctx.dmb_set_bins(dbd, gbd)
    ctx.dmb_set_graph(graph)
    return ctx, dm, gas


def _rel_vec_err(a, b):
    na = np.linalg.norm(b, axis=1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(na, 1e-300 + 1e-30 * na.max())


@pytest.mark.parametrize("fp64", [True, False])
def test_substeps_match_oracle_sequence(fp64):
    w = _w()
    prm, dt = w["params"], w["dt"]
    db, gb = _bins(2000, 1), _bins(2100, 2)
    pairs = pairs_bruteforce(w["dm"], w["gas"], True, prm["box"])
    ctx, dm, gas = _setup(w, db, gb, fp64=fp64)
    sd, sg = _copy(w["dm"]), _copy(w["gas"])
    tv = 1e-12 if fp64 else 1e-5
    for s in (1, 2, 3, 4, 8):
        V_prev = gas["vel"].cpu().numpy()
        sums = ctx.dmb_substep(dm, gas, s, dt)
        ref = oracle_substep(sd, sg, prm, s, dt, db, gb, pairs=pairs)
        assert sums[9] == ref["sums"][9] and sums[10] == ref["sums"][10] and sums[11] == ref["sums"][11]
        assert sums[12] == ref["sums"][12]
        for k in (0, 1, 2, 3, 4, 5, 6, 7, 8, 13):
            tol = 1e-10 if fp64 else 1e-4
            assert abs(sums[k] - ref["sums"][k]) <= tol * (abs(ref["sums"][k]) + 1e-9 * np.abs(ref["sums"][:9]).max()), (s, k)
        ag = ref["active_gas"]
        # transfers of the GPU's own state against the oracle's (the two states differ by rounding)
        dV = gas["vel"].cpu().numpy() - V_prev
        dV_ref = ref["V_new"] - sg["vel"]
        assert np.all(dV[~ag] == 0.0)
        assert np.all(_rel_vec_err(dV[ag], dV_ref[ag]) <= tv), s
        np.testing.assert_allclose(gas["T"].cpu().numpy(), ref["T_new"], rtol=1e-9 if fp64 else 1e-6)
        np.testing.assert_allclose(dm["vel"].cpu().numpy(), ref["mc"]["vel_new"], rtol=0,
                                   atol=(1e-10 if fp64 else 1e-3) * 100.0)
        sd["vel"] = ref["mc"]["vel_new"]
        sg["vel"], sg["T"] = ref["V_new"], ref["T_new"]


def test_graph_replay_matches_direct_launches():
    w = _w()
    db, gb = _bins(2000, 3, top=4), _bins(2100, 4, top=4)
    a = _setup(w, db, gb, graph=False)
    b = _setup(w, db, gb, graph=True)
    for s in (1, 2, 3, 4, 5, 6, 7, 8, 1, 16, 9):   # repeats and a jump: graph reuse and a counter reset
        sa = a[0].dmb_substep(a[1], a[2], s, w["dt"])
        l0 = b[0].dmb_launch_count()
        sb = b[0].dmb_substep(b[1], b[2], s, w["dt"])
        assert b[0].dmb_launch_count() > l0
        assert np.array_equal(sa, sb), s
        for k in ("vel",):
            assert torch.equal(a[1][k], b[1][k]) and torch.equal(a[2][k], b[2][k]), s
        assert torch.equal(a[2]["T"], b[2]["T"])


def test_substep_zero_with_bin_zero_is_the_full_step():
    w = _w()
    n_d, n_g = len(w["dm"]["h"]), len(w["gas"]["h"])
    ctx, dm, gas = _setup(w, np.zeros(n_d, np.uint8), np.zeros(n_g, np.uint8))
    s_sub = ctx.dmb_substep(dm, gas, 0, w["dt"])
    ref_ctx = make_ctx(w)
    dm2, gas2 = device_inputs(w)
    s_full = ref_ctx.dmb_step(dm2, gas2, 0, w["dt"])
    assert torch.equal(dm["vel"], dm2["vel"])
    # the two kick kernels evaluate the same formulas (contraction may differ by an ulp)
    np.testing.assert_allclose(gas["vel"].cpu().numpy(), gas2["vel"].cpu().numpy(), rtol=1e-14, atol=0)
    np.testing.assert_allclose(gas["T"].cpu().numpy(), gas2["T"].cpu().numpy(), rtol=1e-14, atol=0)
    np.testing.assert_allclose(s_sub, s_full, rtol=1e-12, atol=1e-300)


def test_substep_info_and_empty_active_set():
    w = _w()
    db, gb = _bins(2000, 5), _bins(2100, 6)
    db[db == 0] = 1                       # nothing in bin 0: odd substeps move no DM
    gb[gb == 0] = 2
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    ctx, dm, gas = _setup(w, db, gb)
    for s in (0, 1, 2, 4, 6, 12):
        ad, ag = active_mask(db, s), active_mask(gb, s)
        info = ctx.dmb_substep_info(s)
        assert info[0] == ad.sum() and info[1] == ag.sum()
        assert info[3] == np.count_nonzero(ag[pj]) and info[4] == np.count_nonzero(ad[pi])
    v0, V0, T0 = dm["vel"].clone(), gas["vel"].clone(), gas["T"].clone()
    sums = ctx.dmb_substep(dm, gas, 1, w["dt"])
    assert torch.equal(dm["vel"], v0) and torch.equal(gas["vel"], V0) and torch.equal(gas["T"], T0)
    assert np.all(sums == 0.0)


def test_bins_out_of_range_rejected():
    w = _w()
    db = np.zeros(2000, np.uint8)
    db[7] = 64
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    with pytest.raises(dmb.DmbError):
        ctx.dmb_set_bins(_u8(db), _u8(np.zeros(2100, np.uint8)))
    with pytest.raises(dmb.DmbError):
        ctx.dmb_substep(dm, gas, 1, w["dt"])


def test_substeps_with_the_surrogate_epilogue():
    """Substeps with the learned surrogate: the mean field summed inside the tensor-core kernel
    (dmb_set_surrogate_epilogue(1)) against the stored-rates path (the default) on the same state
    (another float32 summation order: 1e-5), and its graph replay against direct launches (bit for
    bit)."""
    w = _w()
    p = w["params"]
    db, gb = _bins(2000, 7), _bins(2100, 8)

    def mk(mode, graph, params=None):
        c = dmb.Context(p["sigma0_cm2"], p["n"], p["m_chi_mp"], p["v0_kms"], p["periodic"], tuple(p["box"]),
                        p["seed"], rate_mode=dmb.DMB_RATE_MLP)
        if params is None:
            c.dmb_train_surrogate(nsamples=1 << 15, epochs=2, seed=5)
        else:
            c.dmb_load_surrogate(params)
        c.dmb_set_surrogate_epilogue(mode)
        dm, gas = device_inputs(w)
        c.dmb_build_grid(dm, gas)
        c.dmb_neighbors()
        c.dmb_set_bins(_u8(db), _u8(gb))
        c.dmb_set_graph(graph)
        return c, dm, gas

    a = mk(1, False)
    params = a[0].dmb_surrogate_params()
    b = mk(1, True, params)
    r = mk(0, False, params)
    V0 = a[2]["vel"].cpu().numpy()
    for s in (1, 2, 3, 4, 8, 1):
        sa = a[0].dmb_substep(a[1], a[2], s, w["dt"])
        sb = b[0].dmb_substep(b[1], b[2], s, w["dt"])
        sr = r[0].dmb_substep(r[1], r[2], s, w["dt"])
        assert np.array_equal(sa, sb), s
        assert torch.equal(a[1]["vel"], b[1]["vel"]) and torch.equal(a[2]["vel"], b[2]["vel"]), s
        assert torch.equal(a[2]["T"], b[2]["T"]), s
        if s == 1:   # same input state in both modes
            dVa = a[2]["vel"].cpu().numpy() - V0
            dVr = r[2]["vel"].cpu().numpy() - V0
            moved = np.linalg.norm(dVr, axis=1) > 0
            assert moved.sum() > 100
            assert np.all(_rel_vec_err(dVa[moved], dVr[moved]) <= 1e-5)
            np.testing.assert_allclose(a[2]["T"].cpu().numpy(), r[2]["T"].cpu().numpy(), rtol=1e-6)

