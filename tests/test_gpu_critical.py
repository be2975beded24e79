"""Critical Reynolds number by the secant method (Section 3) on the GPU
against the oracle, on an 8^3 cosine grid:
* lid parallel to the x sidewall (alpha = 0; tests/golden/critical8.npz,
  tests/golden/make_critical8.py): continuation from rest through Re 500,
  1000, 1400, secant from Re = 1400 and 1500;
* lid parallel to the diagonal plane (alpha = pi/4;
  tests/golden/critical8_diag.npz, tests/golden/make_critical8_diag.py):
  continuation through Re 500, 1000, 1500, secant from Re = 1500 and 1550;
  the leading pair changes between the two starting points (omega ~ 1.73 at
  1500, ~ 4.22 at 1550), and the iteration follows the one that crosses.
Tolerances: Re_cr 1e-5 relative, omega_cr 1e-6 relative, for the FP64,
float-float and mixed forms alike (each secant point moves the grid's Re,
which the captured evaluation graphs of the last two must follow)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402

HERE = os.path.join(os.path.dirname(__file__), "golden")
N = 8
CASES = {"sidewall": ("critical8.npz", 0.0, (500.0, 1000.0, 1400.0), 1400.0, 1500.0),
         "diagonal": ("critical8_diag.npz", np.pi / 4, (500.0, 1000.0, 1500.0), 1500.0, 1550.0)}


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


@pytest.mark.parametrize("case", ["sidewall", "diagonal"])
@pytest.mark.parametrize("prec", ["fp64", "ff", "mixed"])
def test_critical_re_matches_oracle(fv, prec, case):
    fname, alpha, path, re0, re1 = CASES[case]
    gold = np.load(os.path.join(HERE, fname))
    g = fv.Grid(N, N, N, "cosine", alpha=alpha, re=path[0])
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    for re in path:
        g.set_re(re)
        fv.newton_steady(g, U, P, tol=1e-10)
    v0 = torch.tensor(synth.gaussian_velocity((N, N, N), 1), device="cuda")
    re_cr, om, hist = fv.fv_critical_re(g, U, P, v0, re0, re1, rtol=1e-8, prec=prec)
    assert abs(re_cr - float(gold["re_cr"])) <= 1e-5 * re_cr, (re_cr, hist)
    assert abs(om - float(gold["omega_cr"])) <= 1e-6 * om
    assert abs(hist[-1][1]) < 1e-6           # sigma(Re_cr) ~ 0
