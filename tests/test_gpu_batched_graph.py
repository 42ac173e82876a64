"""The batched parameter scan under a captured CUDA graph (dmb_step_batched with
dmb_set_graph(ctx, 1)): the first call runs the step and captures it; later calls replay one
graph per step.  The replayed steps must equal the directly launched ones bit for bit (velocities,
temperatures and the 16 sums), including a step whose pair lists outgrow the captured capacities
(the replay changes nothing, the library regrows its buffers and runs the step again).  The
direct path itself is checked against the oracle box by box in tests/test_gpu_batched.py."""
import numpy as np
import pytest

from gpu_common import require_gpu, torch
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _setup(w, graph, rate=dmb.DMB_RATE_CLOSED):
    p = w["params"]
    ctx = dmb.Context(p["sigma0_cm2"], p["n"], p["m_chi_mp"], p["v0_kms"], True, tuple(p["box"]), p["seed"],
                      rate_mode=rate)
    ctx.dmb_set_graph(graph)
    dm, gas = dmb.to_device(w["dm"]), dmb.to_device(w["gas"])
    db = torch.from_numpy(w["dm_box"].view(np.int32)).cuda()
    gb = torch.from_numpy(w["gas_box"].view(np.int32)).cuda()
    return ctx, dm, gas, db, gb


def _state(dm, gas):
    return [t.clone() for t in (dm["vel"], gas["vel"], gas["T"])]


def test_replayed_steps_equal_direct_steps():
    w = W.boxes_workload(nbox=7, n_lo=600, n_hi=6000, seed=91, dt=2e-3)
    ref = _setup(w, False)
    gra = _setup(w, True)
    launches = []
    for step in range(6):
        s_ref = ref[0].dmb_step_batched(ref[1], ref[3], ref[2], ref[4], w["boxes"], step, w["dt"])
        l0 = gra[0].dmb_launch_count()
        s_gra = gra[0].dmb_step_batched(gra[1], gra[3], gra[2], gra[4], w["boxes"], step, w["dt"])
        launches.append(gra[0].dmb_launch_count() - l0)
        torch.cuda.synchronize()
        assert np.array_equal(s_ref, s_gra), (step, s_ref - s_gra)
        for a, b in zip(_state(ref[1], ref[2]), _state(gra[1], gra[2])):
            assert torch.equal(a, b), step
    assert s_ref[9] > 0 and s_ref[12] > 0
    # steps after the first replay the same graph: its launches are counted as the kernels it holds
    assert len(set(launches[2:])) == 1


def test_overflow_of_the_captured_lists_repeats_the_step():
    w = W.boxes_workload(nbox=4, n_lo=2000, n_hi=4000, seed=92, dt=2e-3)
    ref = _setup(w, False)
    gra = _setup(w, True)
    for step in range(2):        # capture, then one replay
        ref[0].dmb_step_batched(ref[1], ref[3], ref[2], ref[4], w["boxes"], step, w["dt"])
        gra[0].dmb_step_batched(gra[1], gra[3], gra[2], gra[4], w["boxes"], step, w["dt"])
    # the caller grows h in place: about 1.7x the pairs, beyond the captured capacities (h stays
    # below a quarter of the box side, as the periodic boxes require)
    for c in (ref, gra):
        c[1]["h"].mul_(1.2)
        c[2]["h"].mul_(1.2)
    assert float(ref[1]["h"].max() + ref[2]["h"].max()) < 0.5
    for step in range(2, 5):     # overflow and repeat, recapture, replay
        s_ref = ref[0].dmb_step_batched(ref[1], ref[3], ref[2], ref[4], w["boxes"], step, w["dt"])
        s_gra = gra[0].dmb_step_batched(gra[1], gra[3], gra[2], gra[4], w["boxes"], step, w["dt"])
        torch.cuda.synchronize()
        assert np.array_equal(s_ref, s_gra), step
        for a, b in zip(_state(ref[1], ref[2]), _state(gra[1], gra[2])):
            assert torch.equal(a, b), step


def test_replay_with_the_surrogate_and_the_quadrature():
    w = W.boxes_workload(nbox=3, n_lo=800, n_hi=3000, seed=93, dt=2e-3)
    for rate in (dmb.DMB_RATE_QUAD, dmb.DMB_RATE_MLP):
        ref = _setup(w, False, rate)
        gra = _setup(w, True, rate)
        if rate == dmb.DMB_RATE_MLP:
            ref[0].dmb_train_surrogate(nsamples=1 << 15, epochs=2, seed=3)
            gra[0].dmb_load_surrogate(ref[0].dmb_surrogate_params())
        for step in range(3):
            s_ref = ref[0].dmb_step_batched(ref[1], ref[3], ref[2], ref[4], w["boxes"], step, w["dt"])
            s_gra = gra[0].dmb_step_batched(gra[1], gra[3], gra[2], gra[4], w["boxes"], step, w["dt"])
            torch.cuda.synchronize()
            assert np.array_equal(s_ref, s_gra), (rate, step)
            for a, b in zip(_state(ref[1], ref[2]), _state(gra[1], gra[2])):
                assert torch.equal(a, b), (rate, step)
