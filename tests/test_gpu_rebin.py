"""dmb_rebin_dm (timestep feedback from Eq. prob_criterion): bit-exact against the oracle's rule
on random and edge-case ratios, and end to end: after rebinning, the Monte Carlo at each
particle's new timestep has every criterion ratio <= 1, and each ratio is the old one scaled
by exactly 2^(b' - b) (P_ij is proportional to dt)."""
import numpy as np
import pytest

from oracle.substep import rebin
from paper_2603_24688_gb300 import workloads as W
from gpu_common import device_inputs, make_ctx, require_gpu, torch

pytestmark = pytest.mark.gpu


def test_rebin_matches_the_oracle():
    require_gpu()
    rng = np.random.default_rng(9)
    n = 100_003
    x = (10.0 ** rng.uniform(-4, 5, n)).astype(np.float32)
    x[:64] = np.float32(2.0) ** rng.integers(-6, 12, 64).astype(np.float32)
    x[64:70] = [0.0, 1.0, 0.25, np.inf, np.nan, -1.0]
    b = rng.integers(0, 20, n).astype(np.uint8)
    act = rng.integers(0, 2, n).astype(np.uint8)
    w = W.box_workload(n_dm=64, n_gas=64, seed=3)
    ctx = make_ctx(w)
    for substep, max_bin, use_act in ((0, 19, False), (12, 19, True), (4096, 7, True), (0, 63, False)):
        xd = torch.from_numpy(x).cuda()
        bd = torch.from_numpy(b.copy()).cuda()
        ad = torch.from_numpy(act).cuda() if use_act else None
        moved = ctx.dmb_rebin_dm(xd, bd, max_bin, substep, ad)
        ref = rebin(x, b, max_bin, substep, act.astype(bool) if use_act else None)
        got = bd.cpu().numpy()
        assert np.array_equal(got, ref)
        assert moved == int(np.count_nonzero(ref != b))
    with pytest.raises(Exception):
        ctx.dmb_rebin_dm(torch.zeros(4, dtype=torch.float32, device="cuda"),
                         torch.zeros(4, dtype=torch.uint8, device="cuda"), 64)


def test_rebinned_timesteps_meet_the_criterion():
    require_gpu()
    # at dt = 2^6 dt_min most particles of the 1 barn box break the criterion (ratios of order 10),
    # so the new bins spread over the lower ones
    w = W.box_workload(n_dm=8192, n_gas=8192, sigma0_cm2=1e-24, seed=21)
    ctx = make_ctx(w)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    nd = len(w["dm"]["h"])
    dt_min, B = 1e-4, 6

    def ratios(dt):
        vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
        pr = torch.empty(nd, dtype=torch.float32, device="cuda")
        ctx.dmb_mc_scatter_dm(11, dt, vel, None, None, pr, None)
        return pr

    r0 = ratios(dt_min * 2 ** B)
    h0 = r0.cpu().numpy()
    assert np.mean(h0 > 1.0) > 0.5
    bins = torch.full((nd,), B, dtype=torch.uint8, device="cuda")
    ctx.dmb_rebin_dm(r0, bins, B, 0)
    nb = bins.cpu().numpy().astype(int)
    assert np.array_equal(nb, rebin(h0, np.full(nd, B), B, 0).astype(int))
    for bb in np.unique(nb):
        sel = nb == bb
        hb = ratios(dt_min * 2 ** int(bb)).cpu().numpy()
        # exact scaling by a power of two, and the criterion met (bin 0 is as small as it goes)
        assert np.array_equal(hb[sel], (h0[sel] * np.float32(2.0) ** np.float32(int(bb) - B)).astype(np.float32))
        if bb > 0:
            assert np.all(hb[sel] <= 1.0)
            # and the bin is the largest that meets it
            demoted = sel & (h0 > 1.0)
            assert np.all(h0[demoted] * 2.0 ** (int(bb) + 1 - B) > 1.0)
