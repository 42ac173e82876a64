"""Oracle parity of the benchmark's own configuration: the 8M DM + 2M gas galaxy with
sigma = sigma0 (v / 100 km/s)^n for n in {-4, -2, 0, 2}, the gas mean field from the learned
surrogate (the timed path: k_mlp_tc then k_meanfield) and from the closed forms, and the Monte
Carlo, on sampled particles that the FP64 oracle evaluates one by one (Eqs. gas-dVdt, gas-dTdt
with the App. B closed forms; Eqs. dm-update-vels, dm-update-prob, scatter_chi).

Tolerances.  Closed form: 1e-5 relative, as the other float32 tests.  Surrogate: each pair's FA
and FB carry the network's relative error, so a gas row's transfer can be off by at most
eps_A sum_i |cA t_i FA_i w_i| (and likewise for du/dt with eps_B); eps_A, eps_B are the worst
relative errors the training itself measured on its held-out points (against the float64 device
quadrature), plus the quadrature's own 1e-5.  The rows' median error must also stay below the
1e-3 rate-error target.  Pairs outside the training box fall back to quadrature and are counted.
"""
import numpy as np
import pytest

from gpu_common import device_inputs, require_gpu, torch
from oracle import mlp as O
from oracle import units
from oracle.mc import mc_scatter
from oracle.meanfield import meanfield_gas, pair_rates
from oracle.pairs import pairs_bruteforce
from paper_2603_24688_gb300 import dmb
from paper_2603_24688_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NS = (-4, -2, 0, 2)


@pytest.fixture(scope="module")
def galaxy():
    require_gpu()
    w = W.named("galaxy10M")
    dm, gas = device_inputs(w)
    # the bench's surrogate: one network for every n of the scan
    p = w["params"]
    tctx = dmb.Context(p["sigma0_cm2"], -2, p["m_chi_mp"], p["v0_kms"], False, (0.0, 0.0, 0.0), p["seed"],
                       rate_mode=dmb.DMB_RATE_MLP)
    rep = tctx.dmb_train_surrogate(nsamples=1 << 21, epochs=128, seed=11)   # the bench's recipe
    params = tctx.dmb_surrogate_params()
    tctx.close()
    rng = np.random.default_rng(30)
    gsample = rng.choice(len(w["gas"]["h"]), 24, replace=False)
    gpi, gpj = pairs_bruteforce(w["dm"], w["gas"], False, None, gas_subset=gsample, block=200000)
    r = np.linalg.norm(w["dm"]["pos"], axis=1)
    near = np.nonzero((np.abs(w["dm"]["pos"][:, 2]) < 1.0) & (r < 15.0))[0]
    dsample = rng.choice(near, 40, replace=False)
    dpi, dpj = pairs_bruteforce(w["dm"], w["gas"], False, None, dm_subset=dsample, block=4)
    return dict(w=w, dm=dm, gas=gas, report=rep, params=params, gsample=gsample, gpairs=(gpi, gpj),
                dsample=dsample, dpairs=(dpi, dpj))


def _meanfield(g, n, mode):
    w = g["w"]
    p = dict(w["params"], n=n)
    ctx = dmb.Context(p["sigma0_cm2"], n, p["m_chi_mp"], p["v0_kms"], False, (0.0, 0.0, 0.0), p["seed"],
                      rate_mode=mode)
    if mode == dmb.DMB_RATE_MLP:
        ctx.dmb_load_surrogate(g["params"])
    ctx.dmb_build_grid(g["dm"], g["gas"])
    npairs = ctx.dmb_neighbors()
    nb = len(w["gas"]["h"])
    acc = torch.empty((nb, 3), dtype=torch.float64, device="cuda")
    dudt = torch.empty(nb, dtype=torch.float64, device="cuda")
    ctx.dmb_meanfield_gas(acc, dudt)
    fb = ctx.dmb_surrogate_fallbacks() if mode == dmb.DMB_RATE_MLP else 0
    torch.cuda.synchronize()
    s = g["gsample"]
    out = acc[torch.from_numpy(s).cuda()].cpu().numpy(), dudt[torch.from_numpy(s).cuda()].cpu().numpy(), (fb, npairs)
    ctx.close()
    return out, p


def _oracle_rows(g, p):
    """Oracle transfers of the sampled gas rows and the absolute sums that bound a relative rate error."""
    w = g["w"]
    pi, pj = g["gpairs"]
    acc, dudt = meanfield_gas(w["dm"], w["gas"], pi, pj, p)
    gg, wv, A, B = pair_rates(w["dm"], w["gas"], pi, pj, p)
    mu = w["gas"]["mu"][pj]
    coef = w["dm"]["mass"][pi] * units.MSUN_PER_MP / (p["m_chi_mp"] + mu) * gg
    nb = len(w["gas"]["h"])
    sA = np.zeros((nb, 3))
    for c in range(3):
        np.add.at(sA[:, c], pj, np.abs(coef * A * wv[:, c]))
    sUA = np.zeros(nb)
    np.add.at(sUA, pj, np.abs(coef * A * np.sum(wv * wv, axis=1)))
    sUB = np.zeros(nb)
    np.add.at(sUB, pj, np.abs(coef * mu / (p["m_chi_mp"] + mu) * B))
    s = g["gsample"]
    return acc[s], dudt[s], sA[s], sUA[s], sUB[s]


@pytest.mark.parametrize("n", NS)
def test_surrogate_meanfield_against_the_oracle(galaxy, n):
    rep = galaxy["report"]
    eps_a, eps_b = float(rep[1]) + 1e-5, float(rep[2]) + 1e-5     # worst held-out error + quadrature's
    (a_got, u_got, (fb, npairs)), p = _meanfield(galaxy, n, dmb.DMB_RATE_MLP)
    a_ref, u_ref, sA, sUA, sUB = _oracle_rows(galaxy, p)
    assert np.all(np.abs(a_got - a_ref) <= eps_a * sA + 1e-5 * np.abs(a_ref) + 1e-300)
    assert np.all(np.abs(u_got - u_ref) <= eps_a * sUA + eps_b * sUB + 1e-5 * np.abs(u_ref) + 1e-300)
    rel = np.linalg.norm(a_got - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    print(f"n = {n}: fallbacks {fb}, acc relative error median {np.median(rel):.2e} max {rel.max():.2e}; "
          f"eps_A {eps_a:.2e} eps_B {eps_b:.2e}")
    assert np.median(rel) < 1e-3
    assert 0 <= fb < 0.01 * npairs


def test_bench_network_meets_the_rate_error_target(galaxy):
    """The bench's network (its recipe, one network for the whole scan) at the 1e-3 target on the
    worst case: on its held-out points against the float64 device quadrature, and, independently
    of the quadrature, against the oracle's closed forms (App. B) over the training box's whole s
    range at the galaxy's tau and m_chi, through the tensor-core engine that evaluates the pairs."""
    rep = galaxy["report"]
    assert rep[1] <= 1e-3 and rep[2] <= 1e-3, rep[:5]
    w = galaxy["w"]
    p = w["params"]
    ctx = dmb.Context(p["sigma0_cm2"], -2, p["m_chi_mp"], p["v0_kms"], False, (0.0, 0.0, 0.0), p["seed"],
                      rate_mode=dmb.DMB_RATE_MLP)
    ctx.dmb_load_surrogate(galaxy["params"])
    s = np.logspace(-2, 2, 801)
    hot = w["gas"]["T"] > 0
    tau = units.varsigma2_kms2(w["gas"]["T"][hot], w["gas"]["mu"][hot]) / p["v0_kms"] ** 2
    for n in NS:
        for t in np.unique(tau)[:4]:
            X = O.inputs(s, t * np.ones_like(s), p["m_chi_mp"], n).astype(np.float32)
            Y = torch.empty((len(s), 2), dtype=torch.float32, device="cuda")
            ctx.dmb_surrogate_infer_tc(torch.from_numpy(X).cuda(), Y)
            FA, FB = O.rates_from_outputs(Y.cpu().numpy().astype(np.float64), s, n)
            FAr, FBr = O.rates_from_outputs(O.targets(s, n), s, n)
            eA, eB = np.abs(FA / FAr - 1), np.abs(FB / FBr - 1)
            print(f"n = {n}, tau = {t:.3e}: FA worst {eA.max():.2e}, FB worst {eB.max():.2e}")
            assert eA.max() <= 1e-3 and eB.max() <= 1e-3, (n, t, eA.max(), eB.max())
    ctx.close()


@pytest.mark.parametrize("n", NS)
def test_closed_form_meanfield_against_the_oracle(galaxy, n):
    (a_got, u_got, _), p = _meanfield(galaxy, n, dmb.DMB_RATE_CLOSED)
    a_ref, u_ref, sA, sUA, sUB = _oracle_rows(galaxy, p)
    err = np.linalg.norm(a_got - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    assert np.all(err < 1e-5), err.max()
    assert np.all(np.abs(u_got - u_ref) <= 1e-5 * (np.abs(u_ref) + 1e-3 * np.abs(u_ref).max()))


@pytest.mark.parametrize("n", NS)
def test_monte_carlo_against_the_oracle(galaxy, n):
    w = galaxy["w"]
    p = dict(w["params"], n=n)
    ctx = dmb.Context(p["sigma0_cm2"], n, p["m_chi_mp"], p["v0_kms"], False, (0.0, 0.0, 0.0), p["seed"])
    ctx.dmb_build_grid(galaxy["dm"], galaxy["gas"])
    ctx.dmb_neighbors()
    nd = len(w["dm"]["h"])
    vel = torch.empty((nd, 3), dtype=torch.float64, device="cuda")
    sc = torch.empty(nd, dtype=torch.uint8, device="cuda")
    pa = torch.empty(nd, dtype=torch.int32, device="cuda")
    pt = torch.empty(nd, dtype=torch.float64, device="cuda")
    dt = 2e-3
    ctx.dmb_mc_scatter_dm(7, dt, vel, sc, pa, None, pt)
    torch.cuda.synchronize()
    s = galaxy["dsample"]
    idx = torch.from_numpy(s).cuda()
    got_v, got_s = vel[idx].cpu().numpy(), sc[idx].cpu().numpy().astype(bool)
    got_p = pa[idx].cpu().numpy().view(np.uint32).astype(np.uint64)
    got_t = pt[idx].cpu().numpy()
    ctx.close()
    pi, pj = galaxy["dpairs"]
    out = mc_scatter(w["dm"], w["gas"], pi, pj, p, 7, dt)
    np.testing.assert_allclose(got_t, out["C_total"][s], rtol=2e-5)
    band = out["gap"][s] <= 1e-6
    mism = (got_s != out["scattered"][s]) | (got_p != out["partner"][s])
    assert not np.any(mism & ~band)
    ok = out["scattered"][s] & ~mism
    dv = got_v[ok] - w["dm"]["vel"][s][ok]
    dv_ref = out["vel_new"][s][ok] - w["dm"]["vel"][s][ok]
    assert np.all(np.linalg.norm(dv - dv_ref, axis=1) <= 1e-5 * np.linalg.norm(dv_ref, axis=1) + 1e-9)
