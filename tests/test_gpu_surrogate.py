"""The learned rate surrogate on the GPU: forward and gradients against the CPU reference,
training on device-quadrature data, and the mean field with the surrogate against the oracle."""
import time

import numpy as np
import pytest

from gpu_common import device_inputs, require_gpu, torch
from oracle import mlp as O
from oracle.meanfield import meanfield_gas
from oracle.pairs import pairs_bruteforce
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _ctx(n=0, mode=dmb.DMB_RATE_MLP, w=None):
    w = w or W.box_workload(n_dm=64, n_gas=64, n=n)
    p = w["params"]
    return dmb.Context(p["sigma0_cm2"], n, p["m_chi_mp"], p["v0_kms"], True, p["box"], p["seed"], rate_mode=mode)


def test_forward_matches_cpu_reference():
    rng = np.random.default_rng(3)
    p = (rng.uniform(-1, 1, O.NPARAM) * 0.2).astype(np.float32)
    ctx = _ctx()
    ctx.dmb_load_surrogate(p)
    X = rng.uniform(-1, 1, (1000, 4)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty((1000, 2), dtype=torch.float32, device="cuda")
    ctx.dmb_surrogate_infer(Xd, Yd)
    got = Yd.cpu().numpy()
    ref, _ = O.forward(p.astype(np.float64), X.astype(np.float64), bf16_ops=True)
    assert np.max(np.abs(got - ref)) < 2e-3 * (1 + np.abs(ref).max())


def test_gradients_match_cpu_reference():
    rng = np.random.default_rng(4)
    p = (rng.uniform(-1, 1, O.NPARAM) * 0.2).astype(np.float32)
    ctx = _ctx()
    ctx.dmb_load_surrogate(p)
    B = 512
    X = rng.uniform(-1, 1, (B, 4)).astype(np.float32)
    Y = rng.normal(size=(B, 2)).astype(np.float32)
    g = torch.empty(O.NPARAM, dtype=torch.float32, device="cuda")
    loss = ctx.dmb_surrogate_grad(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), g)
    gl = g.cpu().numpy().astype(np.float64)
    ref_loss, ref = O.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), bf16_ops=True)
    assert abs(loss - ref_loss) < 1e-3 * ref_loss
    k = 0
    for name, shape in O.SIZES:
        n = int(np.prod(shape))
        a, b = gl[k:k + n], ref[k:k + n]
        k += n
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel < 2e-2 and cos > 0.9998, (name, rel, cos)


@pytest.fixture(scope="module")
def trained():
    ctx = _ctx(0)
    t0 = time.time()
    rep = ctx.dmb_train_surrogate(nsamples=1 << 20, epochs=24, seed=7)
    return dict(ctx=ctx, report=rep, params=ctx.dmb_surrogate_params(), seconds=time.time() - t0)


def test_training_reaches_the_accuracy_target(trained):
    rep = trained["report"]
    print("surrogate report", rep.tolist())
    # validation against the device quadrature
    assert rep[3] < 1e-3 and rep[4] < 1e-3          # mean relative error of FA, FB
    assert rep[1] < 2e-2 and rep[2] < 2e-2          # worst case over 1e5 held-out points


@pytest.mark.parametrize("n", [-4, -2, 0, 2])
def test_trained_network_against_closed_forms(trained, n):
    # independent of the device quadrature: the oracle's closed forms (App. B)
    s = np.logspace(-1.9, 1.9, 2000)
    X = O.inputs(s, 0.05 * np.ones_like(s), 2.0, n).astype(np.float32)
    ctx = trained["ctx"]
    Yd = torch.empty((len(s), 2), dtype=torch.float32, device="cuda")
    ctx.dmb_surrogate_infer(torch.from_numpy(X).cuda(), Yd)
    FA, FB = O.rates_from_outputs(Yd.cpu().numpy().astype(np.float64), s, n)
    T = O.targets(s, n)
    FAr, FBr = O.rates_from_outputs(T, s, n)
    eA, eB = np.abs(FA / FAr - 1), np.abs(FB / FBr - 1)
    print(f"n={n}: FA max {eA.max():.2e} mean {eA.mean():.2e}; FB max {eB.max():.2e} mean {eB.mean():.2e}")
    assert eA.mean() < 1e-3 and eB.mean() < 1e-3
    assert eA.max() < 1e-2 and eB.max() < 1e-2


def test_meanfield_with_surrogate_against_oracle(trained):
    # the box workload (gas at T = 1e4 K: tau = 8.3e-3 is inside the training box)
    w = W.named("box4k")
    ctx = _ctx(0, w=w)
    ctx.dmb_load_surrogate(trained["params"])
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    nb = len(w["gas"]["h"])
    acc = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(nb, dtype=torch.float64, device="cuda")
    ctx.dmb_meanfield_gas(acc, dudt)
    fb = ctx.dmb_surrogate_fallbacks()
    pi, pj = pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    a_ref, u_ref = meanfield_gas(w["dm"], w["gas"], pi, pj, w["params"])
    a = acc.cpu().numpy()
    err = np.linalg.norm(a - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    print("surrogate mean field: max rel err", err.max(), "fallbacks", fb)
    assert err.max() < 3e-3
    u = dudt.cpu().numpy()
    scale = np.abs(u_ref) + 1e-3 * np.abs(u_ref).max()
    assert np.max(np.abs(u - u_ref) / scale) < 3e-3
    assert fb < 0.01 * len(pi)


def test_surrogate_requires_weights_and_known_n():
    w = W.box_workload(n_dm=700, n_gas=700, n=1)
    ctx = _ctx(1, w=w)
    dm, gas = device_inputs(w)
    ctx.dmb_build_grid(dm, gas)
    ctx.dmb_neighbors()
    acc = torch.empty((700, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(700, dtype=torch.float64, device="cuda")
    with pytest.raises(dmb.DmbError) as e:
        ctx.dmb_meanfield_gas(acc, dudt)
    assert e.value.status == dmb.DMB_ERR_STATE
