"""16^3 lid-driven cube at Re = 1000 (lid parallel to the x sidewall, cosine
grid): Newton steady state from rest (continuation in Re) and the 5 leading
eigenvalues by implicitly restarted Arnoldi (Krylov dimension 30, Philox
Gaussian start vector of seed 1), against the stored oracle result
(tests/golden/config1_16.npz, written by tests/golden/make_config1.py).

Tolerances: steady velocity max-rel 1e-9; eigenvalues |dlam| <= 1e-7 |lam|
(real and imaginary parts compared through the complex difference)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden", "config1_16.npz")
N = 16


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1704_08521_gb300 as m
    return m


def _steady(fv, prec):
    g = fv.Grid(N, N, N, "cosine", alpha=0.0, re=200.0)
    U = torch.zeros(g.n_vel, dtype=torch.float64, device="cuda")
    P = torch.zeros(g.n_cell, dtype=torch.float64, device="cuda")
    hist = []
    for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
        g.set_re(re)
        st = fv.newton_steady(g, U, P, tol=1e-10, prec=prec)
        hist.append((re, st["iterations"], st["res_final"], st["gmres_total"]))
    return g, U, P, hist


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_config1_newton_matches_oracle(fv, prec):
    gold = np.load(GOLD)
    g, U, P, hist = _steady(fv, prec)
    torch.cuda.synchronize()
    u = U.cpu().numpy()
    ref = gold["U"]
    assert np.abs(u - ref).max() / np.abs(ref).max() < 1e-9, hist
    assert hist[-1][2] < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "ff"])
def test_config1_arnoldi_matches_oracle(fv, prec):
    gold = np.load(GOLD)
    g = fv.Grid(N, N, N, "cosine", alpha=0.0, re=1000.0)
    U = torch.tensor(gold["U"], device="cuda")
    v0 = torch.tensor(synth.gaussian_velocity((N, N, N), 1), device="cuda")
    evec = torch.empty(2 * g.n_vel, dtype=torch.float64, device="cuda")
    lam, info = fv.arnoldi_leading(g, U, v0, m=30, nev=5, evec=evec, prec=prec)
    lam = np.array(lam)
    ref = gold["lam"]
    for l in lam:                   # as sets: conjugate ordering may differ
        d = np.min(np.abs(ref - l))
        assert d <= 1e-7 * abs(l), (lam, ref)
    # leading eigenvector agrees up to the normalisation (unit W-norm, phase)
    e = evec.cpu().numpy()
    z = e[:g.n_vel] + 1j * e[g.n_vel:]
    zr = gold["evec0"] + 1j * gold["evec0_imag"]
    c = np.vdot(zr, z) / np.vdot(zr, zr)
    assert np.abs(z - c * zr).max() < 1e-5 * np.abs(zr).max()
