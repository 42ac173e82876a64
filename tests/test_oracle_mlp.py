"""Pins for the CPU reference of the surrogate network (finite differences, envelopes)."""
import math

import numpy as np

from oracle import mlp as O
from oracle.hyp1f1 import hyp1f1_neg


def _params(seed=0):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-1, 1, O.NPARAM) * 0.15
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params()
    X = rng.uniform(-1, 1, (64, 4))
    Y = rng.normal(size=(64, 2))
    loss, g = O.loss_and_grad(p, X, Y, bf16_ops=False)
    idx = rng.choice(O.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [0, 512, 640, 17000, 33000, O.NPARAM - 1]])
    for k in idx:
        e = np.zeros_like(p)
        e[k] = 1e-6
        fd = (O.loss_and_grad(p + e, X, Y, False)[0] - O.loss_and_grad(p - e, X, Y, False)[0]) / 2e-6
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 0.0])
    r = O.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125 and r[4] == 0.0
    assert abs(r[3] + 3.140625) < 1e-12


def test_envelopes_carry_the_limits():
    # the residual targets vanish at x -> 0 and as x -> infinity (DLMF 13.7.2)
    for n in (-4, -2, 0, 2):
        t = O.targets(np.array([1e-4, 3e3]), n)
        assert np.all(np.abs(t) < 2e-3), (n, t)
        eA, eB = O.envelope(n)
        for env, a, b in ((eA, -(n + 1) / 2, 2.5), (eB, -(n + 3) / 2, 1.5)):
            # large x: the power law Gamma(b)/Gamma(b-a) x^-a
            x = 1e6
            assert abs(hyp1f1_neg(a, b, x) / np.exp(O.log_envelope(env, x)) - 1) < 1e-5
            # small x: the first two Taylor coefficients, so the residual is third order (a wrong
            # p leaves O(x) = 1e-3, a wrong q O(x^2) = 1e-6 at x = 1e-3)
            for x in (1e-3, 2e-3):
                res = np.log(hyp1f1_neg(a, b, x)) - O.log_envelope(env, x)
                assert abs(res) < 3e-8 * (x / 1e-3) ** 3, (n, a, x, res)
            # the cubic inside the envelope has no root on x >= 0
            p, q, r, m = env
            assert p > 0 and q >= 0 and r > 0 and m != 0


def test_round_trip_rates():
    s = np.array([0.3, 2.0, 40.0])
    for n in (-2, 2):
        y = O.targets(s, n)
        FA, FB = O.rates_from_outputs(y, s, n)
        x = 0.5 * s * s
        for k in range(3):
            assert abs(FA[k] / hyp1f1_neg(-(n + 1) / 2, 2.5, x[k]) - 1) < 1e-12
            assert abs(FB[k] / hyp1f1_neg(-(n + 3) / 2, 1.5, x[k]) - 1) < 1e-12
