"""Critical Reynolds number by the secant method (Section 3) on the GPU
against the oracle (tests/golden/critical8.npz, tests/golden/make_critical8.py):
8^3 cosine grid, alpha = 0, steady states by continuation from rest, secant
from Re = 1400 and 1500 on the real part of the leading eigenvalue.
Tolerances: Re_cr 1e-5 relative, omega_cr 1e-6 relative, for the FP64,
float-float and mixed forms alike (each secant point moves the grid's Re,
which the captured evaluation graphs of the last two must follow)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "critical8.npz")
N = 8


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


@pytest.mark.parametrize("prec", ["fp64", "ff", "mixed"])
def test_critical_re_matches_oracle(fv, prec):
    gold = np.load(GOLD)
    g = fv.Grid(N, N, N, "cosine", alpha=0.0, re=500.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    for re in (500.0, 1000.0, 1400.0):
        g.set_re(re)
        fv.newton_steady(g, U, P, tol=1e-10)
    v0 = torch.tensor(synth.gaussian_velocity((N, N, N), 1), device="cuda")
    re_cr, om, hist = fv.fv_critical_re(g, U, P, v0, 1400.0, 1500.0, rtol=1e-8, prec=prec)
    assert abs(re_cr - float(gold["re_cr"])) <= 1e-5 * re_cr, (re_cr, hist)
    assert abs(om - float(gold["omega_cr"])) <= 1e-6 * om
    assert abs(hist[-1][1]) < 1e-6           # sigma(Re_cr) ~ 0
