"""Launch shapes and their autotuner: the physics does not depend on the shapes (same pair
set, same Monte Carlo, mean field equal up to the float32 summation order), the tuner picks
from its candidate lists, and out-of-range shapes are refused."""
import numpy as np
import pytest

from gpu_common import device_inputs, gpu_pairs, require_gpu, torch
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def wl():
    w = W.subsample(W.named("galaxy1M", n=-2), 150_000, 60_000, seed=4)
    return w


def _ctx(w, mlp_params=None):
    p = w["params"]
    mode = dmb.DMB_RATE_MLP if mlp_params is not None else dmb.DMB_RATE_CLOSED
    c = dmb.Context(p["sigma0_cm2"], p["n"], p["m_chi_mp"], p["v0_kms"], False, p["box"], p["seed"], rate_mode=mode)
    if mlp_params is not None:
        c.dmb_load_surrogate(mlp_params)
    return c


def _run(ctx, w):
    dm, gas = device_inputs(w)
    pi, pj = gpu_pairs(ctx, dm, gas)
    ng, nd = len(w["gas"]["h"]), len(w["dm"]["h"])
    acc = torch.empty((ng, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(ng, dtype=torch.float64, device="cuda")
    ctx.dmb_meanfield_gas(acc, dudt)
    vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
    ctx.dmb_mc_scatter_dm(3, w["dt"], vel, sc)
    order = np.lexsort((pi, pj))
    return pi[order], pj[order], acc.cpu().numpy(), dudt.cpu().numpy(), vel.cpu().numpy(), sc.cpu().numpy()


@pytest.fixture(scope="module")
def surrogate():
    w = W.box_workload(n_dm=64, n_gas=64, n=-2)
    p = w["params"]
    c = dmb.Context(p["sigma0_cm2"], -2, p["m_chi_mp"], p["v0_kms"], True, p["box"], p["seed"],
                    rate_mode=dmb.DMB_RATE_MLP)
    c.dmb_train_surrogate(nsamples=1 << 18, epochs=4, seed=5)
    return c.dmb_surrogate_params()


@pytest.mark.parametrize("mlp", [False, True])
def test_results_do_not_depend_on_shapes(wl, surrogate, mlp):
    params = surrogate if mlp else None
    ref = _run(_ctx(wl, params), wl)
    for shapes in ({"unit": 16, "seg": 512, "mf_blocks_per_sm": 8, "mc_blocks_per_sm": 4, "tc_warpgroups": 2},
                   {"unit": 128, "seg": 4096, "mf_blocks_per_sm": 32, "mc_blocks_per_sm": 16, "tc_warpgroups": 4}):
        ctx = _ctx(wl, params)
        ctx.dmb_set_shapes(shapes)
        assert ctx.dmb_get_shapes() == shapes
        got = _run(ctx, wl)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])     # the pair set
        assert np.array_equal(got[4], ref[4]) and np.array_equal(got[5], ref[5])     # the Monte Carlo
        na = np.linalg.norm(ref[2], axis=1)
        err = np.linalg.norm(got[2] - ref[2], axis=1) / np.maximum(na, 1e-300)
        assert np.all(err[na > 0] < 1e-5)
        scale = np.abs(ref[3]) + 1e-6 * np.abs(ref[3]).max()
        assert np.max(np.abs(got[3] - ref[3]) / scale) < 1e-5


def test_autotune_picks_candidates_and_keeps_pairs(wl, surrogate):
    ctx = _ctx(wl, surrogate)
    dm, gas = device_inputs(wl)
    shapes, times = ctx.dmb_autotune(dm, gas)
    assert shapes["unit"] in (16, 32, 64, 128)
    assert shapes["seg"] in (512, 1024, 2048, 4096)
    assert shapes["mf_blocks_per_sm"] in (8, 16, 32)
    assert shapes["mc_blocks_per_sm"] in (4, 8, 16, 32)
    assert shapes["tc_warpgroups"] in (2, 3, 4)
    assert len(times) == 23 and all(t > 0 for t in times)
    # the grid and pairs are left built: the mean field runs without a new search
    ng = len(wl["gas"]["h"])
    acc = torch.empty((ng, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(ng, dtype=torch.float64, device="cuda")
    ctx.dmb_meanfield_gas(acc, dudt)
    assert torch.isfinite(acc).all()


def test_shapes_out_of_range_refused(wl):
    ctx = _ctx(wl)
    bad = {"unit": 2, "seg": 2048, "mf_blocks_per_sm": 32, "mc_blocks_per_sm": 32, "tc_warpgroups": 3}
    with pytest.raises(dmb.DmbError):
        ctx.dmb_set_shapes(bad)
    bad = {"unit": 64, "seg": 2048, "mf_blocks_per_sm": 32, "mc_blocks_per_sm": 32, "tc_warpgroups": 5}
    with pytest.raises(dmb.DmbError):
        ctx.dmb_set_shapes(bad)


def test_shapes_persist_as_json_keyed_by_workload(wl, tmp_path):
    import json
    path = str(tmp_path / "shapes.json")
    a = _ctx(wl)
    assert a.dmb_load_shapes(path, "galaxy1M-sub") is False          # no file yet
    names = dmb.Context.SHAPE_NAMES
    a.dmb_set_shapes(dict(zip(names, [32, 1024, 16, 8, 3])))
    a.dmb_save_shapes(path, "galaxy1M-sub")
    a.dmb_set_shapes(dict(zip(names, [16, 512, 32, 32, 4])))
    a.dmb_save_shapes(path, "boxes64")
    a.dmb_set_shapes(dict(zip(names, [128, 2048, 8, 4, 2])))
    a.dmb_save_shapes(path, "galaxy1M-sub")                           # replaces its own entry only
    stored = json.load(open(path))
    assert stored == {"galaxy1M-sub": [128, 2048, 8, 4, 2], "boxes64": [16, 512, 32, 32, 4]}
    b = _ctx(wl)
    assert b.dmb_load_shapes(path, "boxes64") is True
    assert [b.dmb_get_shapes()[k] for k in names] == [16, 512, 32, 32, 4]
    assert b.dmb_load_shapes(path, "other") is False
    with pytest.raises(dmb.DmbError):
        b.dmb_save_shapes(path, "bad key/with slash")
    json.dump({"x": [1, 2, 3, 4, 5]}, open(path, "w"))               # out of range: refused
    with pytest.raises(dmb.DmbError):
        b.dmb_load_shapes(path, "x")
