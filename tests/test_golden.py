"""The stored small-Gram oracle values (tests/golden/gram_small_oracle.txt,
written by tests/golden/make_golden.py from oracle/ alone): the oracle still
reproduces them, and the stored straight-line values converge to the true
kernel I_0(2 sqrt<a,b>) (the Riemann function of the constant-coefficient
Goursat problem, Appendix A) at the scheme's rate 4 per dyadic order (Sec. 3.1),
a check that does not run the scheme."""
import os

import numpy as np

import oracle
from paper_2006_14794_gb300 import inputs
from tests import truth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gram_small_oracle.txt")


def load():
    gram, lines = {}, {}
    for row in open(GOLDEN):
        if row.startswith("#") or not row.strip():
            continue
        kind, a, b, v = row.split()
        (gram if kind == "gram" else lines)[(int(a), int(b))] = float(v)
    return gram, lines


def test_oracle_reproduces_the_stored_values():
    w = inputs.gram_small()
    gram, lines = load()
    G = oracle.gram(w["X"], w["Y"], w["dyadic_order"])
    assert len(gram) == G.size
    for (i, j), v in gram.items():
        assert abs(G[i, j] - v) <= 1e-14 * max(1.0, abs(v))
    for lam in range(4):
        k = oracle.pairs(w["lines_x"], w["lines_y"], lam)
        for b in range(k.shape[0]):
            assert abs(k[b] - lines[(b, lam)]) <= 1e-14 * max(1.0, abs(k[b]))


def test_stored_straight_lines_converge_to_the_closed_form():
    w = inputs.gram_small()
    _, lines = load()
    for b in range(w["a"].shape[0]):
        true = truth.series_I0(float(np.dot(w["a"][b], w["b"][b])))
        err = [abs(lines[(b, lam)] - true) for lam in range(4)]
        if err[0] < 1e-12:   # a product too small to show the rate
            continue
        for lam in range(1, 4):   # the error falls about 4x per dyadic order
            assert 3.0 < err[lam - 1] / err[lam] < 5.0
        rich = truth.richardson(lines[(b, 2)], lines[(b, 3)])
        assert abs(rich - true) <= 1e-3 * err[3] + 1e-12
