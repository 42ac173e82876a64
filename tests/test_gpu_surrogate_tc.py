"""The surrogate on the tcgen05 tensor cores (128-row tiles, accumulators in tensor memory)
against the CPU reference of the network and against the warp-level mma.sync engine, for each
warpgroup count: 2 (activations kept in tensor memory as the MMAs' A operand), 3 and 4
(activations in shared memory)."""
import numpy as np
import pytest

from gpu_common import device_inputs, require_gpu, torch, transfer_scales
from oracle import mlp as O
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _ctx(n=0, w=None):
    w = w or W.box_workload(n_dm=64, n_gas=64, n=n)
    p = w["params"]
    return dmb.Context(p["sigma0_cm2"], n, p["m_chi_mp"], p["v0_kms"], True, p["box"], p["seed"],
                       rate_mode=dmb.DMB_RATE_MLP)


def _set_wg(ctx, wg):
    sh = ctx.dmb_get_shapes()
    sh["tc_warpgroups"] = wg
    ctx.dmb_set_shapes(sh)


@pytest.mark.parametrize("wg", [2, 3, 4])
@pytest.mark.parametrize("rows", [1, 200, 128 * 3 * 152 * 2 + 77])
def test_tc_forward_matches_cpu_reference(rows, wg):
    rng = np.random.default_rng(5)
    p = (rng.uniform(-1, 1, O.NPARAM) * 0.2).astype(np.float32)
    ctx = _ctx()
    ctx.dmb_load_surrogate(p)
    _set_wg(ctx, wg)
    X = rng.uniform(-1, 1, (rows, 4)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.full((rows, 2), float("nan"), dtype=torch.float32, device="cuda")
    ctx.dmb_surrogate_infer_tc(Xd, Yd)
    got = Yd.cpu().numpy()
    k = min(rows, 4000)                                 # the CPU reference on a sample
    idx = np.unique(np.concatenate([np.arange(min(rows, 300)), rng.integers(0, rows, k), [rows - 1]]))
    ref, _ = O.forward(p.astype(np.float64), X[idx].astype(np.float64), bf16_ops=True)
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got[idx] - ref)) < 2e-3 * (1 + np.abs(ref).max())
    # the warp-level engine evaluates the same network
    Y2 = torch.empty_like(Yd)
    ctx.dmb_surrogate_infer(Xd, Y2)
    assert np.max(np.abs(got - Y2.cpu().numpy())) < 2e-3 * (1 + np.abs(ref).max())


def test_tc_warpgroup_counts_agree_bit_for_bit():
    """The three kernels issue the same MMAs on the same operands; only where the activations
    live differs, so their outputs are identical."""
    rng = np.random.default_rng(8)
    p = (rng.uniform(-1, 1, O.NPARAM) * 0.2).astype(np.float32)
    ctx = _ctx()
    ctx.dmb_load_surrogate(p)
    rows = 128 * 4 * 152 * 3 + 5
    Xd = torch.from_numpy(rng.uniform(-1, 1, (rows, 4)).astype(np.float32)).cuda()
    out = {}
    for wg in (2, 3, 4):
        _set_wg(ctx, wg)
        Yd = torch.full((rows, 2), float("nan"), dtype=torch.float32, device="cuda")
        ctx.dmb_surrogate_infer_tc(Xd, Yd)
        out[wg] = Yd.cpu().numpy()
    assert np.all(np.isfinite(out[4]))
    assert np.array_equal(out[2], out[4]) and np.array_equal(out[3], out[4])


@pytest.mark.parametrize("wg", [2, 4])
def test_tc_pair_rates_match_the_warp_engine(wg):
    rng = np.random.default_rng(6)
    w = W.subsample(W.named("galaxy1M"), 60_000, 40_000, seed=2)
    w["params"]["n"] = -2
    p = w["params"]
    ctx = dmb.Context(p["sigma0_cm2"], -2, p["m_chi_mp"], p["v0_kms"], False, p["box"], p["seed"],
                      rate_mode=dmb.DMB_RATE_MLP)
    ctx.dmb_train_surrogate(nsamples=1 << 18, epochs=4, seed=3)
    _set_wg(ctx, wg)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    npairs = ctx.dmb_neighbors()
    assert npairs > 100_000
    nb = len(w["gas"]["h"])
    out = {}
    for eng in (0, 1):
        ctx.dmb_set_surrogate_engine(eng)
        acc = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
        dudt = torch.empty(nb, dtype=torch.float64, device="cuda")
        ctx.dmb_meanfield_gas(acc, dudt)
        out[eng] = (acc.cpu().numpy(), dudt.cpu().numpy(), ctx.dmb_surrogate_fallbacks())
    a0, u0, f0 = out[0]
    a1, u1, f1 = out[1]
    assert f0 == f1
    na = np.linalg.norm(a1, axis=1)
    err = np.linalg.norm(a0 - a1, axis=1) / np.maximum(na, 1e-30)
    assert np.all(err[na > 0] < 2e-3), err.max()
    scale = np.abs(u1) + 1e-3 * np.abs(u1).max()
    assert np.max(np.abs(u0 - u1) / scale) < 2e-3


def _modes(ctx, w, nb):
    """The gas mean field with the rates stored (mode 0) and summed in the epilogue (mode 1)."""
    out = {}
    for mode in (0, 1):
        ctx.dmb_set_surrogate_epilogue(mode)
        acc = torch.full((nb, 3), float("nan"), dtype=torch.float64, device="cuda")
        dudt = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.dmb_meanfield_gas(acc, dudt)
        out[mode] = (acc.cpu().numpy(), dudt.cpu().numpy(), ctx.dmb_surrogate_fallbacks())
    return out


def _gpu_pairs(ctx):
    n = ctx.dmb_neighbors()
    pairs = torch.empty((n, 2), dtype=torch.int32, device="cuda")
    ctx.dmb_neighbors(pairs)
    pp = pairs.cpu().numpy().view(np.uint32).astype(np.int64)
    return pp[:, 0], pp[:, 1]


@pytest.mark.parametrize("wg", [2, 3, 4])
@pytest.mark.parametrize("where", ["galaxy", "box"])
def test_mean_field_in_the_epilogue_matches_stored_rates(wg, where):
    """dmb_set_surrogate_epilogue(1) forms each pair's overlap and rates inside the tensor-core
    kernel and sums the pair terms per gas row over each warp's 32 pairs; mode 0 (the default)
    stores the rates for k_meanfield.  The rates and pair terms are the same, the float32
    summation order differs: every gas row agrees within 1e-5 of the sums of its absolute pair
    terms (Eqs. gas-dVdt, gas-dTdt), and the fallback counts are equal."""
    if where == "galaxy":
        w = W.subsample(W.named("galaxy1M"), 60_000, 40_000, seed=2)
        w["params"]["n"] = -2
    else:   # periodic box: the minimum image inside the epilogue, and cold gas rows
        w = W.box_workload(n_dm=6000, n_gas=5000, seed=41, n=-2)
        w["gas"]["T"][::7] = 0.0
    p = w["params"]
    ctx = dmb.Context(p["sigma0_cm2"], -2, p["m_chi_mp"], p["v0_kms"], p["periodic"], tuple(p["box"]), p["seed"],
                      rate_mode=dmb.DMB_RATE_MLP)
    ctx.dmb_train_surrogate(nsamples=1 << 18, epochs=4, seed=3)
    _set_wg(ctx, wg)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    pi, pj = _gpu_pairs(ctx)
    assert len(pi) > 50_000
    nb = len(w["gas"]["h"])
    out = _modes(ctx, w, nb)
    (a0, u0, f0), (a1, u1, f1) = out[0], out[1]
    assert f0 == f1
    assert np.all(np.isfinite(a1)) and np.all(np.isfinite(u1))
    sa, su = transfer_scales(w, pi, pj, dict(p, n=-2))
    assert np.all(np.abs(a1 - a0) <= 1e-5 * sa), np.max(np.abs(a1 - a0) / np.maximum(sa, 1e-300))
    assert np.all(np.abs(u1 - u0) <= 1e-5 * su), np.max(np.abs(u1 - u0) / np.maximum(su, 1e-300))
    # gas particles without partners get exact zeros in both modes
    lone = np.setdiff1d(np.arange(nb), pj)
    assert np.all(a1[lone] == 0.0) and np.all(u1[lone] == 0.0)


def test_epilogue_mode_argument_checked():
    ctx = _ctx()
    with pytest.raises(dmb.DmbError):
        ctx.dmb_set_surrogate_epilogue(2)
    ctx.dmb_set_surrogate_epilogue(0)
    ctx.dmb_set_surrogate_epilogue(1)

