"""The per-pair Bernoulli variant of the Monte Carlo (dmb_set_mc_variant(ctx, 1)) against the
oracle's sequential restatement (oracle.mc.mc_scatter_bernoulli) on the 4096 + 4096 box: the
scatter decisions and first partners bit-exact outside the 1e-6 band, the new velocities within
the float32 tolerance of the kicks, the sums and ratios as in the categorical variant; once with
the box's dt (sum_j P_ij about 0.02) and once with dt x 100 (about 2 scatters per particle, so
later probabilities follow earlier kicks).  Switching back restores the categorical draw."""
import numpy as np
import pytest

from oracle.kernel import overlap_g_vec
from oracle.mc import mc_scatter, mc_scatter_bernoulli
from oracle.meanfield import pair_geometry
from oracle.pairs import pairs_bruteforce
from paper_2603_24688_gb300 import workloads as W
from gpu_common import device_inputs, make_ctx, require_gpu, torch

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def box():
    w = W.named("box4k")
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    d = pair_geometry(w["dm"], w["gas"], pi, pj, True, w["params"]["box"])
    g = overlap_g_vec(d, w["dm"]["h"][pi], w["gas"]["h"][pj])
    return dict(w=w, pi=pi, pj=pj, g=g)


def _gpu_mc(ctx, w, step, dt):
    nd = len(w["dm"]["h"])
    vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
    pa = torch.empty(nd, dtype=torch.int32, device="cuda")
    pr = torch.empty(nd, dtype=torch.float32, device="cuda")
    pt = torch.empty(nd, dtype=torch.float64, device="cuda")
    ctx.dmb_mc_scatter_dm(step, dt, vel, sc, pa, pr, pt)
    return (vel.cpu().numpy(), sc.cpu().numpy().astype(bool), pa.cpu().numpy().view(np.uint32).astype(np.uint64),
            pr.cpu().numpy(), pt.cpu().numpy())


@pytest.mark.parametrize("dt_scale", [1.0, 100.0])
def test_bernoulli_variant_matches_the_oracle(box, dt_scale):
    require_gpu()
    w = box["w"]
    dt = w["dt"] * dt_scale
    ref = mc_scatter_bernoulli(w["dm"], w["gas"], box["pi"], box["pj"], w["params"], 7, dt, box["g"])
    ctx = make_ctx(w)
    ctx.dmb_set_mc_variant(1)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    v, s, p, pr, pt = _gpu_mc(ctx, w, 7, dt)
    np.testing.assert_allclose(pt, ref["C_total"], rtol=2e-5)
    np.testing.assert_allclose(pr, ref["p_ratio_max"], rtol=2e-5)
    band = ref["gap"] <= 1e-6
    mism = (s != ref["scattered"]) | (p != ref["partner"])
    assert not np.any(mism & ~band), f"{np.count_nonzero(mism & ~band)} decisions differ outside the band"
    assert s.sum() > 10
    if dt_scale > 1:
        assert np.count_nonzero(ref["n_scatter"] >= 2) > 100
    ok = ~mism & ~band
    dv_ref = ref["vel_new"] - w["dm"]["vel"]
    dv = v - w["dm"]["vel"]
    e = np.linalg.norm(dv[ok] - dv_ref[ok], axis=1)
    scale = np.maximum(np.linalg.norm(dv_ref[ok], axis=1), 1.0 * s[ok]) * np.maximum(ref["n_scatter"][ok], 1)
    assert np.all(e <= 10 * TOL32 * scale), e.max()
    assert np.array_equal(v[~s], w["dm"]["vel"][~s])


def test_switching_back_restores_the_categorical_draw(box):
    require_gpu()
    w = box["w"]
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    a = _gpu_mc(ctx, w, 7, w["dt"])
    ctx.dmb_set_mc_variant(1)
    _gpu_mc(ctx, w, 7, w["dt"])
    ctx.dmb_set_mc_variant(0)
    b = _gpu_mc(ctx, w, 7, w["dt"])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    ref = mc_scatter(w["dm"], w["gas"], box["pi"], box["pj"], w["params"], 7, w["dt"], box["g"])
    assert np.array_equal(a[1] | (ref["gap"] <= 1e-6), ref["scattered"] | (ref["gap"] <= 1e-6))
    with pytest.raises(Exception):
        ctx.dmb_set_mc_variant(2)
