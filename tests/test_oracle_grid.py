"""Pins of the oracle grid (Section 3, Eq. 5)."""
import numpy as np
import pytest

from oracle import grid as G


@pytest.mark.parametrize("n", [100, 150, 200, 256])
def test_eq5_step_sizes(n):
    # Section 3: the smallest step (at the wall) is ~0.387/N.  The paper prints
    # ~1.387/N for the largest step (next to x = 0.5); Eq. 5 itself gives
    # 1 + 0.0975 * 2 pi = 1.613/N there (the printed value adds 0.387 instead
    # of 0.613), and the Eq. 5 map is what is implemented.
    ax = G.Axis(n, "sine0975")
    assert abs(ax.dx.min() * n - 0.387) < 2e-3
    assert abs(ax.dx.max() * n - (2.0 - 0.387)) < 2e-3
    assert np.argmin(ax.dx) in (0, n - 1)
    i = int(np.argmax(ax.dx))
    assert min(abs(ax.x[i] - 0.5), abs(ax.x[i + 1] - 0.5)) < 1e-12


@pytest.mark.parametrize("kind", G.MAPS)
def test_symmetry_and_metrics(kind):
    ax = G.Axis(17, kind)
    np.testing.assert_allclose(ax.x + ax.x[::-1], 1.0, atol=1e-15)
    assert np.all(ax.dx > 0)
    np.testing.assert_allclose(ax.dx.sum(), 1.0, atol=1e-15)
    np.testing.assert_allclose(ax.dc.sum(), 1.0, atol=1e-15)     # half cells at walls
    np.testing.assert_allclose(ax.dc[1:-1], 0.5 * (ax.dx[1:] + ax.dx[:-1]), rtol=1e-14)


def test_cosine_closed_form():
    n = 100
    ax = G.Axis(n, "cosine")
    np.testing.assert_allclose(ax.dx[0], 0.5 * (1 - np.cos(np.pi / n)), rtol=1e-12)
    np.testing.assert_allclose(ax.dx[n // 2], 0.5 * (np.cos(np.pi * 50 / n) - np.cos(np.pi * 51 / n)), rtol=1e-12)


def test_volumes():
    g = G.Grid(5, 6, 7, "cosine")
    np.testing.assert_allclose(g.cell_volume().sum(), 1.0, rtol=1e-14)
    for c in range(3):
        np.testing.assert_allclose(g.face_volume(c).sum(), 1.0, rtol=1e-14)
