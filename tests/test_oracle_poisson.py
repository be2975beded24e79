"""Pins of the oracle pressure-correction solver (Section 3, TPF)."""
import numpy as np
import pytest

from oracle import fv, grid as G, poisson


@pytest.mark.parametrize("n", [4, 9, 16])
def test_uniform_neumann_eigenvalues_closed_form(n):
    # uniform Neumann second difference: -(2/h sin(k pi / 2n))^2, k = 0..n-1
    e = poisson.AxisEigen(G.Axis(n, "uniform"))
    h = 1.0 / n
    exact = -(2.0 / h * np.sin(np.arange(n) * np.pi / (2 * n))) ** 2
    np.testing.assert_allclose(np.sort(e.lam), np.sort(exact), atol=1e-9 * n * n)


@pytest.mark.parametrize("kind", G.MAPS)
def test_tpf_solves_DG(kind):
    g = G.Grid(7, 5, 6, kind)
    rng = np.random.default_rng(3)
    r = rng.standard_normal(g.shape_p)
    r -= (r * g.cell_volume()).sum() / g.cell_volume().sum()     # compatible rhs
    phi = poisson.TPF(g).solve(r)
    DG = fv.divergence(g, [fv.gradient(g, phi, c) for c in range(3)])
    np.testing.assert_allclose(DG, r, atol=1e-11 * np.abs(r).max())
    assert abs((phi * g.cell_volume()).sum()) < 1e-13
    np.testing.assert_allclose(poisson.apply_DG(g, phi), DG, atol=1e-10)


def test_null_mode_is_constant():
    e = poisson.AxisEigen(G.Axis(12, "cosine"))
    col = e.E[:, e.null]
    np.testing.assert_allclose(col / col[0], 1.0, rtol=1e-12)
    assert abs(e.lam[e.null]) < 1e-10
    assert np.all(np.delete(e.lam, e.null) < -1.0)
