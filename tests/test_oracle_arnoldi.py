"""Pins of the oracle eigen-solver (Eq. 7, Section 3): the leading eigenvalues
against dense spectra of the same discrete operator."""
import numpy as np
import pytest

from oracle import arnoldi, dense, fv, grid as G, krylov, poisson, simple


def _setup(n, re, alpha, kind="cosine"):
    g = G.Grid(n, n, n, kind)
    tpf = poisson.TPF(g)
    U, P, _ = krylov.newton(g, tpf, re, fv.lid_velocity(alpha))
    return g, tpf, U


def _arnoldi(g, tpf, U, re, nev, m, seed=1):
    wts = fv.pack(fv.weights(g))
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal(wts.size) * (wts > 0)
    x0 = fv.pack(simple.project(g, tpf, fv.unpack(g, x0))[0])
    A = lambda x: fv.pack(simple.shifted_operator(g, tpf, U, fv.unpack(g, x), re, 10.0)[0])
    return arnoldi.arnoldi_leading(A, x0, wts, nev=nev, m=m), A, wts


def _match(lam, ref):
    """max |lam_i - closest ref| (sets, conjugate ordering free)."""
    return max(np.min(np.abs(ref - l)) for l in lam)


def test_dense_constructions_agree():
    g, tpf, U = _setup(5, 150.0, 0.0)
    L = dense.assemble_L(g, U, 150.0)
    a = dense.reduced_spectrum(g, U, 150.0, L)
    b = dense.pencil_spectrum(g, U, 150.0, L)
    assert a.size == b.size == 3 * 4 * 25 - (125 - 1)
    assert _match(a, b) < 1e-9 and _match(b, a) < 1e-9


@pytest.mark.parametrize("n,re,alpha", [(6, 100.0, 0.0), (8, 400.0, 0.0), (6, 300.0, np.pi / 4)])
def test_arnoldi_matches_dense_spectrum(n, re, alpha):
    g, tpf, U = _setup(n, re, alpha)
    ref = dense.reduced_spectrum(g, U, re)
    (lam, X, info), A, wts = _arnoldi(g, tpf, U, re, nev=5, m=30)
    # the five leading eigenvalues, in order, to 1e-10 relative
    np.testing.assert_allclose(lam.real, ref[:5].real, rtol=0, atol=1e-10 * np.abs(ref[0]) + 1e-12)
    np.testing.assert_allclose(np.abs(lam.imag), np.abs(ref[:5].imag), atol=1e-10 * np.abs(ref[0]) + 1e-12)
    for i in range(5):                     # eigen-residual in the W-norm
        x = X[:, i]
        r = A(x.real) + 1j * A(x.imag) - lam[i] * x
        assert np.sqrt(np.sum(wts * np.abs(r) ** 2)) < 1e-8 * abs(lam[i])


def test_stokes_spectrum_real_negative():
    g = G.Grid(6, 6, 6, "cosine")
    tpf = poisson.TPF(g)
    Z = g.zeros_vel()
    # Re = 100 keeps the wanted eigenvalues (~ -0.55, threefold by the cube's
    # symmetry) above -sigma = -10, where the shifted operator parks the
    # gradient complement
    (lam, X, info), _, _ = _arnoldi(g, tpf, Z, 100.0, nev=4, m=24)
    assert np.all(np.abs(lam.imag) < 1e-8 * np.abs(lam.real))
    assert np.all(lam.real < 0)
    ref = dense.reduced_spectrum(g, Z, 100.0)
    np.testing.assert_allclose(lam.real, ref[:4].real, rtol=1e-10)


def test_eigenvector_symmetry_alpha0():
    # the leading mode of the alpha = 0 flow is either even or odd under y -> 1 - y
    g, tpf, U = _setup(6, 100.0, 0.0)
    (lam, X, info), _, _ = _arnoldi(g, tpf, U, 100.0, nev=1, m=20)
    q = fv.unpack(g, X[:, 0].real)
    even = max(np.abs(q[0] - q[0][:, ::-1]).max(), np.abs(q[1] + q[1][:, ::-1]).max())
    odd = max(np.abs(q[0] + q[0][:, ::-1]).max(), np.abs(q[1] - q[1][:, ::-1]).max())
    assert min(even, odd) < 1e-8
