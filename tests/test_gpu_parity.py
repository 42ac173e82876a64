"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (from the accuracy targets of the method): neighbour sets and Monte Carlo
decisions bit-exact except pairs/decisions within 1e-6 relative of the kernel radius or
an acceptance threshold (counted); per-particle transfers within 1e-5 relative in the
float32 path and 1e-12 relative in the float64 path.
"""
import numpy as np
import pytest

from gpu_common import transfer_scales, device_inputs, gpu_pairs, make_ctx, pair_band_mask, require_gpu, torch
from oracle import philox as OP
from oracle.kernel import overlap_g_vec
from oracle.hyp1f1 import hyp1f1_neg_arr
from oracle.mc import mc_scatter
from oracle.meanfield import meanfield_gas, pair_geometry
from oracle.pairs import pairs_bruteforce
from oracle.step import oracle_step
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def box():
    """The 4096 + 4096 periodic box with its oracle pairs, g, mean field and MC."""
    w = W.named("box4k")
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    d = pair_geometry(w["dm"], w["gas"], pi, pj, True, w["params"]["box"])
    g = overlap_g_vec(d, w["dm"]["h"][pi], w["gas"]["h"][pj])
    acc, dudt = meanfield_gas(w["dm"], w["gas"], pi, pj, w["params"], g)
    mc = mc_scatter(w["dm"], w["gas"], pi, pj, w["params"], 7, w["dt"], g)
    return dict(w=w, pi=pi, pj=pj, g=g, acc=acc, dudt=dudt, mc=mc)


def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0, 0, 0, 0x80000000]]
    w = W.named("box4k")
    ctx = make_ctx(w)
    c_dev = torch.from_numpy(ctr.astype(np.uint32).view(np.int32)).cuda()
    out = torch.empty_like(c_dev)
    ctx.dmb_debug_philox(c_dev, out)
    got = out.cpu().numpy().view(np.uint32).astype(np.uint64)
    seed = w["params"]["seed"]
    ref = OP.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], seed & 0xFFFFFFFF, seed >> 32)
    assert np.array_equal(got, np.stack(ref, axis=1))


@pytest.mark.parametrize("fp64", [False, True])
def test_overlap_against_exact(fp64):
    rng = np.random.default_rng(1)
    k = 20000
    hi = rng.uniform(0.03, 1.0, k)
    hj = hi * np.concatenate([rng.uniform(0.0, 1.0, k // 2), rng.uniform(1.0, 30.0, k - k // 2)])
    d = rng.uniform(0.0, 1.0, k) * (hi + hj)
    d[:50] = 0.0
    ref = overlap_g_vec(d, hi, hj)
    ctx = make_ctx(W.named("box4k"), fp64=fp64)
    inp = torch.from_numpy(np.stack([d, hi, hj], 1)).cuda()
    out = torch.empty(k, dtype=torch.float64, device="cuda")
    ctx.dmb_debug_overlap(inp, out)
    got = out.cpu().numpy()
    scale = 1.0 / np.maximum(hi, hj) ** 3        # g h_a^3 is O(1)
    err = np.abs(got - ref) / scale
    if fp64:
        assert np.all(np.abs(got - ref) <= 1e-13 * np.maximum(ref, 1e-3 * scale))
    else:
        # float32 lookup + bicubic interpolation: absolute error in g h_a^3 (an O(1) quantity)
        assert err.max() < 2e-6, err.max()
        big = ref / scale > 0.05
        assert np.max(np.abs(got - ref)[big] / ref[big]) < 2e-5


@pytest.mark.parametrize("n", [-4, -3, -2, -1, 0, 1, 2])
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
def test_rate_integrals(n, fp64, mode):
    from paper_2603_24688_gb300 import dmb
    x = np.concatenate([[0.0, 1e-7, 0.5, 0.999999, 1.0, 1.000001], 10 ** np.linspace(-6, 5, 3000)])
    w = W.box_workload(n_dm=64, n_gas=64, n=n)
    p = w["params"]
    ctx = dmb.Context(p["sigma0_cm2"], n, p["m_chi_mp"], p["v0_kms"], True, p["box"], p["seed"], fp64=fp64,
                      rate_mode=mode)
    out = torch.empty((x.size, 2), dtype=torch.float64, device="cuda")
    ctx.dmb_debug_rates(torch.from_numpy(x).cuda(), out)
    got = out.cpu().numpy()
    refA = hyp1f1_neg_arr(-(n + 1) / 2.0, 2.5, x)
    refB = hyp1f1_neg_arr(-(n + 3) / 2.0, 1.5, x) if n > -3 or n == -4 else np.ones_like(x)
    # closed form: float64 2e-13, float32 4e-6; quadrature (64-point composite Gauss-Legendre,
    # truncation ~2e-8): 5e-8 in float64, 2e-5 in float32
    tol = (2e-13 if fp64 else 4e-6) if mode == 0 else (5e-8 if fp64 else 2e-5)
    np.testing.assert_allclose(got[:, 0], refA, rtol=tol, atol=0)
    np.testing.assert_allclose(got[:, 1], refB, rtol=tol, atol=0)


@pytest.mark.parametrize("fp64", [False, True])
def test_neighbours_box_exact(box, fp64):
    w = box["w"]
    ctx = make_ctx(w, fp64=fp64)
    dm, gas = device_inputs(w)
    gi, gj = gpu_pairs(ctx, dm, gas)
    ref = set(zip(box["pi"].tolist(), box["pj"].tolist()))
    got = set(zip(gi.tolist(), gj.tolist()))
    assert len(got) == len(gi), "duplicate pairs"
    diff = ref ^ got
    if diff:
        a = np.array(sorted(diff))
        assert pair_band_mask(w, a[:, 0], a[:, 1]).all(), f"{len(diff)} pairs differ outside the band"


def _rel_vec_err(got, ref):
    num = np.linalg.norm(got - ref, axis=-1) if got.ndim > 1 else np.abs(got - ref)
    den = np.linalg.norm(ref, axis=-1) if ref.ndim > 1 else np.abs(ref)
    return num / np.maximum(den, 1e-300)


@pytest.mark.parametrize("fp64,mode", [(False, 0), (True, 0), (False, 1), (True, 1)])
def test_meanfield_box(box, fp64, mode):
    from paper_2603_24688_gb300 import dmb
    w = box["w"]
    p = w["params"]
    ctx = dmb.Context(p["sigma0_cm2"], p["n"], p["m_chi_mp"], p["v0_kms"], True, p["box"], p["seed"], fp64=fp64,
                      rate_mode=mode)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    nb = len(w["gas"]["h"])
    acc = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(nb, dtype=torch.float64, device="cuda")
    ctx.dmb_meanfield_gas(acc, dudt)
    a = acc.cpu().numpy()
    u = dudt.cpu().numpy()
    tol = (TOL64 if fp64 else TOL32) if mode == 0 else (5e-8 if fp64 else 2e-5)
    ea = _rel_vec_err(a, box["acc"])
    eu = _rel_vec_err(u, box["dudt"])
    assert np.percentile(ea, 100) < tol, ea.max()
    # heating sums mix signs (w^2 A - e B): bounded by tol times the sum of the absolute terms
    _, su = transfer_scales(w, box["pi"], box["pj"], w["params"], box["g"])
    assert np.all(np.abs(u - box["dudt"]) <= tol * su), np.max(np.abs(u - box["dudt"]) / su)


@pytest.mark.parametrize("fp64", [False, True])
def test_mc_box(box, fp64):
    w = box["w"]
    ref = box["mc"]
    ctx = make_ctx(w, fp64=fp64)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    nd = len(w["dm"]["h"])
    vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
    pa = torch.empty(nd, dtype=torch.int32, device="cuda")
    pr = torch.empty(nd, dtype=torch.float32, device="cuda")
    pt = torch.empty(nd, dtype=torch.float64, device="cuda")
    ctx.dmb_mc_scatter_dm(7, w["dt"], vel, sc, pa, pr, pt)
    v = vel.cpu().numpy()
    s = sc.cpu().numpy().astype(bool)
    p = pa.cpu().numpy().view(np.uint32).astype(np.uint64)
    tol = TOL64 if fp64 else TOL32
    np.testing.assert_allclose(pt.cpu().numpy(), ref["C_total"], rtol=1e-12 if fp64 else 2e-5)
    np.testing.assert_allclose(pr.cpu().numpy(), ref["p_ratio_max"], rtol=2e-5 if not fp64 else 1e-6)
    band = ref["gap"] <= 1e-6
    mism = (s != ref["scattered"]) | (p != ref["partner"])
    assert not np.any(mism & ~band), f"{np.count_nonzero(mism & ~band)} decisions differ outside the band"
    assert s.sum() > 10
    ok = ~mism
    dv_ref = ref["vel_new"] - w["dm"]["vel"]
    dv = v - w["dm"]["vel"]
    e = np.linalg.norm(dv[ok] - dv_ref[ok], axis=1)
    assert np.all(e <= tol * np.maximum(np.linalg.norm(dv_ref[ok], axis=1), 1.0 * s[ok])), e.max()
    # non-scattered particles keep their exact float64 velocity
    assert np.array_equal(v[~s], w["dm"]["vel"][~s])


@pytest.mark.parametrize("fp64", [False, True])
def test_step_box(fp64):
    w = W.named("box4k")
    out = oracle_step(w["dm"], w["gas"], w["params"], 11, w["dt"])
    ctx = make_ctx(w, fp64=fp64)
    dm, gas = device_inputs(w)
    sums = ctx.dmb_step(dm, gas, 11, w["dt"])
    tol = 1e-10 if fp64 else 1e-4
    ref = out["sums"]
    assert sums[12] == ref[12]
    assert sums[9] == ref[9] and sums[10] == ref[10] and sums[11] == ref[11]
    for k in (0, 1, 2, 3, 4, 5, 6, 7, 8, 13, 14):
        assert abs(sums[k] - ref[k]) <= tol * (abs(ref[k]) + 1e-9 * np.abs(ref[:9]).max()), (k, sums[k], ref[k])
    tv = TOL64 if fp64 else TOL32
    dV = gas["vel"].cpu().numpy() - w["gas"]["vel"]
    dV_ref = out["V_new"] - w["gas"]["vel"]
    assert np.all(_rel_vec_err(dV, dV_ref) <= tv)
    np.testing.assert_allclose(gas["T"].cpu().numpy(), out["T_new"], rtol=1e-9 if fp64 else 1e-6)
    # DM: the same decisions outside the 1e-6 band; the kicks of the common scatters within the
    # tolerance of the Monte Carlo test; everyone else keeps the exact float64 velocity
    v = dm["vel"].cpu().numpy()
    mc = out["mc"]
    s_got = np.any(v != w["dm"]["vel"], axis=1)
    band = mc["gap"] <= 1e-6
    assert not np.any((s_got != mc["scattered"]) & ~band)
    both = s_got & mc["scattered"]
    dv, dv_ref = v[both] - w["dm"]["vel"][both], mc["vel_new"][both] - w["dm"]["vel"][both]
    assert np.all(np.linalg.norm(dv - dv_ref, axis=1) <= 10 * tv * np.linalg.norm(dv_ref, axis=1))
    assert np.array_equal(v[~s_got], w["dm"]["vel"][~s_got])
