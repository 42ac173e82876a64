"""The oracle against numbers the paper prints (tests/golden/paper_facts.txt, each with its
passage): the cubic spline's normalisation, support and Plummer equivalence, the constants of
the timestep criterion and its stated cap for m_chi = 2 m_p, and the accuracy the paper states
for its five-term 1F1 expansion, checked against the oracle's own 1F1 (just below x = 50 the
oracle sums the Kummer series, a different formula from the expansion)."""
import math
import os

import numpy as np

from oracle import kernel as K
from oracle import mc as MC
from oracle.hyp1f1 import hyp1f1_neg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.txt")


def _facts():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, val = line.split()[:2]
                out[key] = float(val)
    return out


F = _facts()


def _gl(f, a, b, n=12):
    x, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (b - a) * x + 0.5 * (b + a)
    return 0.5 * (b - a) * float(np.sum(w * f(t)))


def test_spline_integral_support_and_plummer_equivalence():
    h = 1.7
    # piecewise cubic: Gauss-Legendre with 12 nodes is exact on [0, h/2] and [h/2, h]
    mass = sum(_gl(lambda r: 4 * np.pi * r * r * K.W(r, h), a, b) for a, b in ((0, h / 2), (h / 2, h)))
    assert abs(mass - F["spline_integral"]) < 1e-13
    assert K.W(F["spline_support"] * h, h) == 0.0 and K.W(0.999999 * h, h) > 0.0
    # central potential of unit mass smeared by W: -G int W(r) / r d^3r = -4 pi G int W r dr;
    # a Plummer sphere of scale eps has -G / eps there, so h / eps = 4 pi h int_0^h W r dr
    phi0 = sum(_gl(lambda r: 4 * np.pi * r * K.W(r, h), a, b) for a, b in ((0, h / 2), (h / 2, h)))
    assert abs(phi0 * h - F["spline_h_over_plummer_eps"]) < 1e-12


def test_timestep_criterion_constants():
    big = MC.pcap(1e3, 1.0)                                    # (m_chi + mu)/mu large: the 0.1 branch
    assert big == F["prob_cap_large"]
    assert MC.pcap(0.0, 1.0) == F["prob_cap_coefficient"]        # (m_chi + mu)/mu = 1
    # m_chi = 2 m_p: hydrogen (mu = 1) and ionised gas (mu = 0.6); the paper's cap is about 1e-3
    for mu in (1.0, 1.0 / 1.3):
        cap = MC.pcap(2.0, mu)
        assert cap <= 2 * F["prob_cap_mchi2_atmost"] and cap >= 0.5 * F["prob_cap_mchi2_atmost"]


def _expansion(a, b, x, terms):
    """The paper's large-x form of 1F1(a, b; -x), truncated after `terms` terms."""
    s, t = 0.0, 1.0
    for k in range(terms):
        s += t
        t *= (a + k) * (1 + a - b + k) / ((k + 1) * x)
    return math.gamma(b) * x ** (-a) / math.gamma(b - a) * s


def test_five_term_expansion_accuracy_against_the_oracle():
    terms = int(F["hyp1f1_asymptotic_terms"])
    x0 = F["hyp1f1_asymptotic_from_x"]
    tol = F["hyp1f1_asymptotic_rel_err"]
    # the (a, b) of A and B for the paper's power laws (App. B closed forms).  The expansion
    # leaves out a part of order e^-x, negligible from x0 on.  Just below x0 the oracle evaluates
    # the Kummer series instead, a different formula, so that point cross-checks the two.
    for n in (-4, -2, 0, 2):
        for a, b in ((-(n + 1) / 2, 2.5), (-(n + 3) / 2, 1.5)):
            for x in (0.99 * x0, x0, 2 * x0, 1e3, 1e4):
                ref = hyp1f1_neg(a, b, x)
                assert abs(_expansion(a, b, x, terms) / ref - 1) < tol, (n, a, b, x)


def _mass_mp(text):
    val, unit = text.split()
    return {"m_p": 1.0, "GeV": 1.0 / 0.93827208816, "MeV": 1e-3 / 0.93827208816}[unit] * float(val)


def test_box_test_rows_are_the_papers_table():
    from paper_2603_24688_gb300 import boxtest as BT
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "test_params.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                c = [x.strip() for x in line.split("|")]
                npart = [int(x.split("^")[0]) ** int(x.split("^")[1]) if "^" in x else int(float(x)) for x in c[9:11]]
                rows[c[0]] = (_mass_mp(c[1]), float(c[2]), int(c[3]), float(c[4]), float(c[5]), float(c[6]),
                              float(c[7]), float(c[8]), npart[0], npart[1])
    assert set(rows) == set(BT.ROWS)
    for name, want in rows.items():
        got = BT.ROWS[name]
        assert all(abs(a - b) <= 1e-12 * abs(b) for a, b in zip(got, want)), (name, got, want)
