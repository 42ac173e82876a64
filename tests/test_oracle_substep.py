"""Pins for the oracle's hierarchical substep: reduction to the full step, untouched inactive
particles, linearity of every transfer in the particle's own dt, and the activity rule."""
import numpy as np

from oracle.pairs import pairs_bruteforce
from oracle.step import oracle_step
from oracle.substep import active_mask, oracle_substep
from paper_2603_24688_gb300 import workloads as W


def _w():
    return W.box_workload(n_dm=300, n_gas=280, seed=21, n=-2, T_gas=3e4, bulk_dm=(120.0, 0.0, 30.0))


def test_activity_rule():
    b = np.array([0, 1, 2, 3, 11], dtype=np.uint8)
    assert active_mask(b, 0).all()
    assert list(active_mask(b, 1)) == [True, False, False, False, False]
    assert list(active_mask(b, 4)) == [True, True, True, False, False]
    assert list(active_mask(b, 24)) == [True, True, True, True, False]


def test_all_bin_zero_is_the_full_step():
    w = _w()
    dm, gas, prm = w["dm"], w["gas"], w["params"]
    pairs = pairs_bruteforce(dm, gas, True, prm["box"])
    ref = oracle_step(dm, gas, prm, 7, w["dt"], pairs=pairs)
    z = lambda n: np.zeros(n, np.uint8)
    sub = oracle_substep(dm, gas, prm, 7, w["dt"], z(len(dm["h"])), z(len(gas["h"])), pairs=pairs)
    for k in ("acc", "dudt", "V_new", "u_new", "T_new"):
        assert np.array_equal(ref[k], sub[k]), k
    assert np.array_equal(ref["mc"]["vel_new"], sub["mc"]["vel_new"])
    assert np.array_equal(ref["mc"]["scattered"], sub["mc"]["scattered"])
    np.testing.assert_allclose(sub["sums"], ref["sums"], rtol=1e-13, atol=0)


def test_inactive_particles_untouched_and_dt_linearity():
    w = _w()
    dm, gas, prm = w["dm"], w["gas"], w["params"]
    pairs = pairs_bruteforce(dm, gas, True, prm["box"])
    rng = np.random.default_rng(3)
    db = rng.integers(0, 4, len(dm["h"])).astype(np.uint8)
    gb = rng.integers(0, 4, len(gas["h"])).astype(np.uint8)
    s = 6                                   # bins 0 and 1 active
    sub = oracle_substep(dm, gas, prm, s, w["dt"], db, gb, pairs=pairs)
    ad, ag = sub["active_dm"], sub["active_gas"]
    assert np.array_equal(ad, db <= 1) and np.array_equal(ag, gb <= 1)
    assert np.array_equal(sub["mc"]["vel_new"][~ad], dm["vel"][~ad])
    assert np.array_equal(sub["V_new"][~ag], gas["vel"][~ag])
    assert np.array_equal(sub["T_new"][~ag], gas["T"][~ag])
    # the same particles with every bin 0: transfers of bin-1 particles are exactly twice as large
    z = oracle_substep(dm, gas, prm, s, w["dt"], np.zeros_like(db), np.zeros_like(gb), pairs=pairs)
    g1 = gb == 1
    np.testing.assert_allclose(sub["V_new"][g1] - gas["vel"][g1], 2.0 * (z["V_new"][g1] - gas["vel"][g1]),
                               rtol=1e-12, atol=1e-300)
    pi = pairs[0]
    P_sub = sub["mc"]["P"]
    P_all = z["mc"]["P"][ad[pi]]
    scale = 2.0 ** db[pi[ad[pi]]].astype(float)
    np.testing.assert_allclose(P_sub, scale * P_all, rtol=1e-14)


def test_rebin_rule_against_brute_force():
    """The new bin is the largest b' <= b whose scaled ratio ratio 2^(b' - b) is <= 1 (found by
    trying every bin), promotions happen only below 1/4, at a boundary of the larger step and
    under max_bin, and inactive particles keep their bins."""
    from oracle.substep import rebin
    rng = np.random.default_rng(5)
    n = 4000
    b = rng.integers(0, 12, n)
    x = (10.0 ** rng.uniform(-3, 4, n)).astype(np.float32)
    x[:40] = np.float32(2.0) ** rng.integers(-4, 10, 40).astype(np.float32)     # exact powers of two
    x[40:45] = [0.0, 1.0, 0.25, np.inf, np.nan]
    for substep, max_bin in ((0, 11), (8, 11), (0, 5), (3, 63)):
        act = rng.integers(0, 2, n).astype(bool)
        nb = rebin(x, b, max_bin, substep, act)
        for i in range(n):
            if not act[i]:
                assert nb[i] == b[i]
                continue
            xi = float(x[i])
            if not np.isfinite(xi):
                assert nb[i] == 0
            elif xi > 1.0:
                ok = [c for c in range(int(b[i]) + 1) if xi * 2.0 ** (c - int(b[i])) <= 1.0]
                assert nb[i] == (max(ok) if ok else 0), (xi, b[i], nb[i])
            elif xi < 0.25 and b[i] < max_bin and substep % (1 << (int(b[i]) + 1)) == 0:
                assert nb[i] == b[i] + 1 and xi * 2.0 <= 0.5
            else:
                assert nb[i] == b[i]
