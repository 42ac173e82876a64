"""Pins for the oracle's pair set: brute force vs literal loops and the cell list."""
import itertools

import numpy as np

from oracle import pairs as Pr
from paper_2603_24688_gb300 import workloads as W


def _literal(dm, gas, periodic, box):
    out = []
    for i, j in itertools.product(range(len(dm["h"])), range(len(gas["h"]))):
        d = 0.0
        for c in range(3):
            x = dm["pos"][i, c] - gas["pos"][j, c]
            if periodic:
                while x > box[c] / 2:
                    x -= box[c]
                while x < -box[c] / 2:
                    x += box[c]
            d += x * x
        if d ** 0.5 < dm["h"][i] + gas["h"][j]:
            out.append((i, j))
    return out


def _tiny(seed, n=40, periodic=True):
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 1.3, 0.8])
    mk = lambda: dict(pos=rng.uniform(0, 1, (n, 3)) * box, h=rng.uniform(0.02, 0.3, n))
    return mk(), mk(), box


def test_bruteforce_equals_literal_periodic_and_open():
    for seed, periodic in ((1, True), (2, False), (3, True)):
        dm, gas, box = _tiny(seed, periodic=periodic)
        pi, pj = Pr.pairs_bruteforce(dm, gas, periodic, box)
        assert list(zip(pi.tolist(), pj.tolist())) == _literal(dm, gas, periodic, box)


def test_strict_inequality_at_contact():
    dm = dict(pos=np.array([[0.0, 0.0, 0.0]]), h=np.array([0.25]))
    gas = dict(pos=np.array([[0.5, 0.0, 0.0], [0.4999999, 0, 0]]), h=np.array([0.25, 0.25]))
    pi, pj = Pr.pairs_bruteforce(dm, gas, False, None)
    assert pj.tolist() == [1]


def test_celllist_equals_bruteforce_on_box():
    w = W.box_workload(n_dm=1500, n_gas=1300, L=2.0, seed=77)
    a = Pr.pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    b = Pr.pairs_celllist(w["dm"], w["gas"], True, w["params"]["box"])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_subset_query_matches_full():
    w = W.box_workload(n_dm=800, n_gas=900, seed=5)
    full_i, full_j = Pr.pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"])
    sub = np.array([3, 100, 799])
    si, sj = Pr.pairs_bruteforce(w["dm"], w["gas"], True, w["params"]["box"], dm_subset=sub)
    mask = np.isin(full_i, sub)
    assert np.array_equal(si, full_i[mask]) and np.array_equal(sj, full_j[mask])
