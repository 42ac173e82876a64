"""Confluent hypergeometric function 1F1(a, b; -x), x >= 0 (oracle, FP64).

Sec. 2.4 evaluates 1F1 at small a, b and negative argument by combining Kummer's
transformation (DLMF 13.2.39) with the large-argument expansion (DLMF 13.7.2):
    1F1(a, b; -x) = Gamma(b) x^(-a) / Gamma(b - a) * sum_k (a)_k (1 + a - b)_k / (k! x^k)
used for x >= 50; below that the paper calls GSL.  Here, below x = 50, Kummer's
transformation 1F1(a, b; -x) = e^(-x) 1F1(b - a, b; x) is summed as a power series:
for the arguments the method uses (b - a = (n + 6)/2 > 0, b > 0) every term is
positive, so the sum has no cancellation.

Reading: the paper truncates the large-x sum at five terms.  For even n the
series terminates (1 + a - b is a non-positive integer) within five terms and
five terms are exact; for other n the oracle keeps adding terms until they fall
below 1e-17 of the sum (or the terms start to grow), which is at least as
accurate as five terms.

Parity: pinned.  tests/test_oracle_rates.py checks against mpmath.hyp1f1 at
high precision over x in [0, 1e4] and against the erf special case
1F1(1/2, 3/2; -x) = (sqrt(pi)/2) erf(sqrt(x)) / sqrt(x), and the continuity of
the two branches at the x = 50 seam.
"""
import math

import numpy as np

X_SWITCH = 50.0


def _kummer_series(a, b, x):
    """e^(-x) * sum_k (b-a)_k x^k / ((b)_k k!)   (DLMF 13.2.39 then 13.2.2)."""
    c = b - a
    term = 1.0
    total = 1.0
    k = 0
    while True:
        term *= (c + k) * x / ((b + k) * (k + 1.0))
        total += term
        k += 1
        if term < 1e-17 * total and k > x:
            break
        if k > 100000:
            raise RuntimeError("1F1 series did not converge")
    return math.exp(-x) * total


def _asymptotic(a, b, x):
    """Gamma(b) x^-a / Gamma(b-a) * sum_k (a)_k (1+a-b)_k / (k! x^k)   (DLMF 13.7.2)."""
    e = 1.0 + a - b
    term = 1.0
    total = 1.0
    k = 0
    prev = float("inf")
    while True:
        term *= (a + k) * (e + k) / ((k + 1.0) * x)
        k += 1
        if term == 0.0:
            break
        if abs(term) > prev:  # asymptotic series started to diverge
            break
        total += term
        prev = abs(term)
        if abs(term) < 1e-17 * abs(total) and k >= 5:
            break
    lg = math.lgamma(b) - math.lgamma(b - a)
    sign = math.copysign(1.0, math.gamma(b)) * math.copysign(1.0, math.gamma(b - a))
    return sign * math.exp(lg - a * math.log(x)) * total


def hyp1f1_neg(a, b, x):
    """1F1(a, b; -x) for scalar x >= 0."""
    x = float(x)
    if x < 0.0:
        raise ValueError("x must be >= 0")
    if not b - a > 0.0:
        raise ValueError("only b - a > 0 is used by the method")
    if x == 0.0:
        return 1.0
    if x < X_SWITCH:
        return _kummer_series(a, b, x)
    return _asymptotic(a, b, x)


def hyp1f1_neg_vec(a, b, x):
    """Elementwise hyp1f1_neg over an array of x (a Python loop)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(x.shape)
    flat = out.reshape(-1)
    for k, xv in enumerate(x.reshape(-1)):
        flat[k] = hyp1f1_neg(a, b, xv)
    return out


def hyp1f1_neg_arr(a, b, x):
    """Vectorised hyp1f1_neg: the same two branches, iterated on arrays.

    Below X_SWITCH the positive Kummer series is summed until every element's
    term is below 1e-17 of its sum (and past k > x); above it the large-x
    series adds terms while they decrease, stopping per element as in the
    scalar version.
    """
    if not b - a > 0.0:
        raise ValueError("only b - a > 0 is used by the method")
    x = np.asarray(x, dtype=np.float64)
    out = np.ones(x.shape)
    small = (x > 0.0) & (x < X_SWITCH)
    if np.any(small):
        xs = x[small]
        c = b - a
        term = np.ones_like(xs)
        total = np.ones_like(xs)
        k = 0
        while True:
            term = term * (c + k) * xs / ((b + k) * (k + 1.0))
            total = total + term
            k += 1
            if k > xs.max() and np.all(term < 1e-17 * total):
                break
        out[small] = np.exp(-xs) * total
    large = x >= X_SWITCH
    if np.any(large):
        xl = x[large]
        e = 1.0 + a - b
        term = np.ones_like(xl)
        total = np.ones_like(xl)
        prev = np.full_like(xl, np.inf)
        active = np.ones(xl.shape, dtype=bool)
        k = 0
        while np.any(active) and k < 200:
            term = term * (a + k) * (e + k) / ((k + 1.0) * xl)
            k += 1
            stop = (term == 0.0) | (np.abs(term) > prev)
            active &= ~stop
            total = np.where(active, total + term, total)
            prev = np.where(active, np.abs(term), prev)
            active &= ~((np.abs(term) < 1e-17 * np.abs(total)) & (k >= 5))
        lg = math.lgamma(b) - math.lgamma(b - a)
        sign = math.copysign(1.0, math.gamma(b)) * math.copysign(1.0, math.gamma(b - a))
        out[large] = sign * np.exp(lg - a * np.log(xl)) * total
    return out
