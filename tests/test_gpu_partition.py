"""Spatial decomposition on the GPU: each slab's library run (owned + ghost particles) gives its
owned particles the same Monte Carlo (bit for bit where the coordinate frame is the same) and
the same mean field (to the summation order) as the run over all particles."""
import numpy as np
import pytest

from gpu_common import device_inputs, make_ctx, require_gpu, torch
from paper_2603_24688_gb300 import partition as PT
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _run(w, dm_np, gas_np, fp64):
    ctx = make_ctx(w, fp64=fp64)
    wl = dict(w, dm=dm_np, gas=gas_np)
    dm, gas = device_inputs(wl)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    ng, nd = len(gas_np["h"]), len(dm_np["h"])
    acc = torch.empty((ng, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(ng, dtype=torch.float64, device="cuda")
    ctx.dmb_meanfield_gas(acc, dudt)
    vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
    pa = torch.empty(nd, dtype=torch.int32, device="cuda")
    ctx.dmb_mc_scatter_dm(9, w["dt"], vel, sc, pa)
    return acc.cpu().numpy(), dudt.cpu().numpy(), vel.cpu().numpy(), sc.cpu().numpy(), pa.cpu().numpy()


@pytest.mark.parametrize("which,fp64", [("open", False), ("open", True), ("periodic", False)])
def test_slabs_reproduce_the_whole_step(which, fp64):
    w = (W.galaxy_workload(30000, 20000, seed=W.SEED_BASE + 79, n=-2) if which == "open"
         else W.box_workload(n_dm=6000, n_gas=5000, seed=80, n=0, bulk_dm=(80.0, 0.0, 0.0)))
    prm = w["params"]
    full = _run(w, w["dm"], w["gas"], fp64)
    x = np.concatenate([w["dm"]["pos"][:, 0], w["gas"]["pos"][:, 0]])
    if prm["periodic"]:
        x = np.mod(x, prm["box"][0])
    edges = PT.slab_edges(x, 3)
    tol = 1e-12 if fp64 else 1e-5
    for r in range(3):
        v = PT.rank_view(w["dm"], w["gas"], edges, r, prm["periodic"], prm["box"])
        loc = _run(w, PT.subset(w["dm"], v["dm"]), PT.subset(w["gas"], v["gas"]), fp64)
        od, og = v["dm"][v["dm_owned"]], v["gas"][v["gas_owned"]]
        mo, go = v["dm_owned"], v["gas_owned"]
        same = (loc[3][mo] == full[3][od]) & (loc[4][mo] == full[4][od])
        if fp64 or prm["periodic"]:
            # the same coordinate frame (float64, or the periodic box's): bit for bit
            assert same.all()
        else:
            # float32 with a slab's own coordinate frame: distances differ in the last bits, so a
            # draw within ~1e-7 of its threshold may fall the other way
            assert np.count_nonzero(~same) <= max(1, 1e-4 * len(od))
        assert np.array_equal(loc[2][mo][same], full[2][od][same])   # Monte Carlo velocities
        na = np.linalg.norm(full[0][og], axis=1)
        err = np.linalg.norm(loc[0][go] - full[0][og], axis=1) / np.maximum(na, 1e-300)
        assert np.all(err[na > 0] <= tol), err.max()
        scale = np.abs(full[1][og]) + 1e-6 * np.abs(full[1][og]).max()
        assert np.max(np.abs(loc[1][go] - full[1][og]) / scale) <= tol
