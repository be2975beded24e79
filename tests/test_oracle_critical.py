"""Pins of the Richardson extrapolation and the secant search."""
import json
import os

import numpy as np
import pytest

from oracle import critical

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table3.json")


@pytest.mark.parametrize("case", ["alpha0", "alpha45"])
def test_richardson_reproduces_table3(case):
    # Table 3: the bold rows are the Richardson values of consecutive grids
    d = json.load(open(GOLD))
    N = d["grids"]
    for key, rkey, tol in (("re_cr", "richardson_re", 0.015), ("omega_cr", "richardson_omega", 2e-5)):
        for i in range(1, 4):
            x = critical.richardson(N[i - 1], d[case][key][i - 1], N[i], d[case][key][i])
            assert abs(x - d[case][rkey][i]) <= tol, (case, key, i, x)


def test_richardson_exact_for_quadratic_error():
    f = lambda n: 3.25 + 7.0 / n ** 2
    assert abs(critical.richardson(40, f(40), 60, f(60)) - 3.25) < 1e-13


def test_secant_closed_form():
    # sigma(Re) = 1e-3 (Re - 1919.37) (Re + 50) / 2000: root 1919.37
    root, extra, hist = critical.secant(lambda r: ((r - 1919.37) * (r + 50) / 2e6, r), 1800.0, 2000.0, rtol=1e-10)
    assert abs(root - 1919.37) < 1e-6
    assert extra == root
