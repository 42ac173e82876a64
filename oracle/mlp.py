"""CPU reference of the rate surrogate network (test infrastructure, float64 numpy).

The paper has no surrogate (it evaluates 1F1, Sec. 2.4); this module restates the network the
library trains, so that the GPU forward and backward kernels can be checked element by
element: a 4 -> 128 -> 128 -> 128 -> 2 MLP with the squared ReLU act(z) = max(z, 0)^2 as its
activation, parameters packed as
W1[128][4] b1 W2[128][128] b2 W3[128][128] b3 W4[2][128] b4.  The GPU feeds the two
128 x 128 layers bf16 operands (weights and activations rounded to nearest even) and
accumulates in float32; `forward(..., bf16=True)` applies the same roundings in float64.

Targets (what the network learns): with x = s^2/2 and the App. B closed forms
FA = 1F1(-(n+1)/2, 5/2; -x), FB = 1F1(-(n+3)/2, 3/2; -x), the outputs are log F - log E for
each, against the envelope E = (1 + p x + q x^2 + r x^3)^m of F = 1F1(a, b; -x), e = -a, m = e/3:
r from the large-x limit 1F1(a, b; -x) -> Gamma(b)/Gamma(b-a) x^-a (DLMF 13.7.2), p and q from
the series 1 + (e/b) x + e(e-1)/(2b(b+1)) x^2 + ... (DLMF 13.2.2), q kept >= 0; E = 1 for e = 0.

Parity: pinned by finite differences of this module's own loss (tests/test_oracle_mlp.py)
and by the closed-form targets being the pinned oracle rates.
"""
import math

import numpy as np

from .hyp1f1 import hyp1f1_neg_arr

H = 128
SIZES = [("W1", (H, 4)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
         ("W4", (2, H)), ("b4", (2,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([d[name].reshape(-1) for name, _ in SIZES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def act(z):
    """Squared ReLU, max(z, 0)^2."""
    r = np.maximum(z, 0.0)
    return r * r


def act_grad(z):
    """d act / dz = 2 max(z, 0) (continuous, so the loss is once differentiable everywhere)."""
    return 2.0 * np.maximum(z, 0.0)


def forward(p, X, bf16_ops=True):
    """Return (y, cache) for inputs X [N, 4]."""
    d = unpack(p)
    r = bf16 if bf16_ops else (lambda v: np.asarray(v, dtype=np.float64))
    z1 = X @ d["W1"].T + d["b1"]
    a1 = r(act(z1))
    z2 = a1 @ r(d["W2"]).T + d["b2"]
    a2 = r(act(z2))
    z3 = a2 @ r(d["W3"]).T + d["b3"]
    a3 = act(z3)
    y = a3 @ d["W4"].T + d["b4"]
    return y, dict(X=X, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, d=d)


def loss_and_grad(p, X, Y, bf16_ops=True):
    """Mean over samples of the summed squared error and its gradient (plain backprop)."""
    y, c = forward(p, X, bf16_ops)
    d = c["d"]
    r = bf16 if bf16_ops else (lambda v: np.asarray(v, dtype=np.float64))
    B = X.shape[0]
    dy = 2.0 * (y - Y) / B
    loss = float(np.sum((y - Y) ** 2) / B)
    g = {}
    g["W4"] = dy.T @ c["a3"]
    g["b4"] = dy.sum(0)
    dz3 = (dy @ d["W4"]) * act_grad(c["z3"])
    dz3r = r(dz3)
    g["W3"] = dz3r.T @ c["a2"]
    g["b3"] = dz3r.sum(0)
    dz2 = (dz3r @ r(d["W3"])) * act_grad(c["z2"])
    dz2r = r(dz2)
    g["W2"] = dz2r.T @ c["a1"]
    g["b2"] = dz2r.sum(0)
    dz1 = (dz2r @ r(d["W2"])) * act_grad(c["z1"])
    g["W1"] = dz1.T @ c["X"]
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def envelope_of(a, b):
    """(p, q, r, m) of the envelope of 1F1(a, b; -x) (module docstring)."""
    e = -a
    if e == 0:
        return 0.0, 0.0, 0.0, 0.0
    m = e / 3.0
    k1, k2 = e / b, e * (e - 1.0) / (2.0 * b * (b + 1.0))
    p = k1 / m
    q = max((k2 - 0.5 * k1 * k1) / m + 0.5 * p * p, 0.0)
    r = (math.gamma(b) / math.gamma(b + e)) ** (1.0 / m)
    return p, q, r, m


def envelope(n):
    """Envelopes of FA and FB at index n: ((p, q, r, m) of FA, (p, q, r, m) of FB)."""
    return envelope_of(-(n + 1) / 2.0, 2.5), envelope_of(-(n + 3) / 2.0, 1.5)


def log_envelope(env, x):
    p, q, r, m = env
    return m * np.log1p(x * (p + x * (q + x * r)))


def inputs(s, tau, m_chi, n):
    return np.stack([0.5 * np.log10(s), 0.5 * np.log10(tau), np.log10(m_chi) * np.ones_like(s),
                     0.25 * n * np.ones_like(s)], axis=1)


def targets(s, n):
    """The network's regression targets from the closed forms (float64)."""
    x = 0.5 * np.asarray(s, dtype=np.float64) ** 2
    FA = hyp1f1_neg_arr(-(n + 1) / 2.0, 2.5, x)
    FB = hyp1f1_neg_arr(-(n + 3) / 2.0, 1.5, x)
    eA, eB = envelope(n)
    return np.stack([np.log(FA) - log_envelope(eA, x), np.log(FB) - log_envelope(eB, x)], axis=1)


def rates_from_outputs(y, s, n):
    x = 0.5 * np.asarray(s, dtype=np.float64) ** 2
    eA, eB = envelope(n)
    return np.exp(y[:, 0] + log_envelope(eA, x)), np.exp(y[:, 1] + log_envelope(eB, x))
