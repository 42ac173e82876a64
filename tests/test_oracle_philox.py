"""Statistical pins for the oracle's Philox4x32-10 streams (no known-answer vectors here)."""
import math

import numpy as np
from scipy import stats

from oracle import philox as P


def test_uniform_conversion_is_exact_in_float32():
    w = np.array([0, 1, 255, 256, 0xFFFFFFFF, 0x80000000], dtype=np.uint64)
    u = P.to_uniform(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert u[0] == 0.5 * 2.0 ** -23 and u[4] == 1.0 - 0.5 * 2.0 ** -23
    r = P.to_uniform52(w, w[::-1])
    assert np.all(r > 0) and np.all(r < 1)
    # k + 0.5 with k < 2^52 is exact in float64: recover k
    k = (r * 2.0 ** 52 - 0.5)
    assert np.all(k == np.floor(k))


def test_outputs_uniform_chi2():
    ids = np.arange(1 << 16, dtype=np.uint64)
    words = P.pair_words(1234, 7, ids, ids[::-1])
    for w in words:
        counts = np.bincount((w >> np.uint64(24)).astype(np.int64), minlength=256)
        chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-4


def test_neighbouring_counters_uncorrelated():
    ids = np.arange(1 << 16, dtype=np.uint64)
    u = P.to_uniform(P.pair_words(99, 3, ids, np.zeros_like(ids))[0])
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / math.sqrt(len(u))
    # different steps and different seeds give unrelated streams
    u2 = P.to_uniform(P.pair_words(99, 4, ids, np.zeros_like(ids))[0])
    u3 = P.to_uniform(P.pair_words(100, 3, ids, np.zeros_like(ids))[0])
    for other in (u2, u3):
        assert abs(np.corrcoef(u, other)[0, 1]) < 5 / math.sqrt(len(u))


def test_counter_is_a_bijection_on_samples():
    # for a fixed key Philox is a permutation of the 128-bit counter space: distinct counters
    # give distinct outputs
    ids = np.arange(1 << 15, dtype=np.uint64)
    w = P.pair_words(5, 0, ids, ids)
    packed = set(zip(*(x.tolist() for x in w)))
    assert len(packed) == len(ids)


def test_streams_are_disjoint():
    # the DM stream sets the top bit of counter word 3, so it never repeats a pair stream
    ids = np.arange(1000, dtype=np.uint64)
    a = P.dm_words(7, 11, ids)
    b = P.pair_words(7, 11, ids, np.zeros_like(ids))
    assert not np.any(a[0] == b[0]) or np.mean(a[0] == b[0]) < 0.01


def test_normals_moments():
    ids = np.arange(1 << 17, dtype=np.uint64)
    z = P.pair_normals(3, 1, ids, ids + np.uint64(17)).reshape(-1)
    n = len(z)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(stats.skew(z)) < 5 * math.sqrt(6 / n)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_direction_isotropic():
    ids = np.arange(1 << 16, dtype=np.uint64)
    r, cth, phi = P.dm_uniforms(8, 2, ids)
    assert stats.kstest(cth, "uniform", args=(-1, 2)).pvalue > 1e-4
    assert stats.kstest(phi, "uniform", args=(0, 2 * math.pi)).pvalue > 1e-4
    assert stats.kstest(r, "uniform").pvalue > 1e-4


def test_deterministic_and_key_dependent():
    ids = np.arange(64, dtype=np.uint64)
    a = P.pair_words(1 << 40, 5, ids, ids)
    b = P.pair_words(1 << 40, 5, ids, ids)
    c = P.pair_words((1 << 40) + 1, 5, ids, ids)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])
