"""Pins of the oracle SIMPLE-like loop (Section 3, Eqs. 8-10)."""
import numpy as np
import pytest

from oracle import fv, grid as G, poisson, simple


def _rand_vel(g, rng):
    return [fv._zero_walls(rng.standard_normal(g.shape_vel(c)), c) for c in range(3)]


def test_exact_solver_stops_after_two_passes():
    g = G.Grid(6, 5, 7, "cosine")
    tpf = poisson.TPF(g)
    w = _rand_vel(g, np.random.default_rng(0))
    v, p, norms = simple.simple_loop(g, w, tpf.solve, eps=1e-8)
    assert len(norms) == 2 and norms[1] < 1e-12 * norms[0]
    v0, p0 = simple.project(g, tpf, w)
    for c in range(3):
        np.testing.assert_allclose(v[c], v0[c], atol=1e-12)


@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_inexact_fp32_solver_reaches_same_fixed_point(omega):
    # Section 3: the loop converges to the fields required by Eqs. 8-9 even
    # when step 1 is solved inexactly (here: the exact solver in float32)
    g = G.Grid(8, 7, 6, "cosine")
    tpf = poisson.TPF(g)
    E = [(e.E.astype(np.float32), e.Einv.astype(np.float32)) for e in tpf.eig]
    inv32 = tpf.inv_den.astype(np.float32)

    def solve32(r):
        a = r.astype(np.float32)
        for d in range(3):
            a = poisson._apply(E[d][1], a, d).astype(np.float32)
        a = a * inv32
        for d in range(3):
            a = poisson._apply(E[d][0], a, d).astype(np.float32)
        return a.astype(np.float64)

    w = _rand_vel(g, np.random.default_rng(1))
    v, p, norms = simple.simple_loop(g, w, solve32, eps=1e-12, omega=omega)
    assert 3 <= len(norms) <= (6 if omega == 1.0 else 60)
    v0, p0 = simple.project(g, tpf, w)
    sc = max(np.abs(x).max() for x in w)
    for c in range(3):
        np.testing.assert_allclose(v[c], v0[c], atol=1e-10 * sc)
    np.testing.assert_allclose(p - (p * g.cell_volume()).sum(), p0, atol=1e-10 * np.abs(p0).max())


def test_wrong_metric_solver_still_converges():
    # a deliberately inexact Poisson solver (exact for the Eq. 5 map with the
    # amplitude 0.08 instead of 0.0975): each pass only contracts the
    # divergence, yet the loop lands on the exact projection
    g = G.Grid(6, 6, 6, "sine0975")
    tpf = poisson.TPF(g)
    gw = G.Grid(6, 6, 6, "sine0975")
    for ax in gw.ax:
        xi = np.arange(ax.n + 1) / ax.n
        ax.x = xi - 0.08 * np.sin(2 * np.pi * xi)
        ax.x[0], ax.x[-1] = 0.0, 1.0
        ax.dx = np.diff(ax.x)
        ax.xc = 0.5 * (ax.x[:-1] + ax.x[1:])
        ax.dc = np.concatenate([[ax.dx[0] / 2], np.diff(ax.xc), [ax.dx[-1] / 2]])
    tw = poisson.TPF(gw)
    w = _rand_vel(g, np.random.default_rng(2))
    v, p, norms = simple.simple_loop(g, w, tw.solve, eps=1e-11, max_pass=400)
    assert len(norms) > 5                       # genuinely iterative
    v0, _ = simple.project(g, tpf, w)
    sc = max(np.abs(x).max() for x in w)
    for c in range(3):
        np.testing.assert_allclose(v[c], v0[c], atol=1e-10 * sc)


def test_shifted_operator_equals_krylov_vector_on_solenoidal_fields():
    g = G.Grid(5, 6, 5, "cosine")
    tpf = poisson.TPF(g)
    rng = np.random.default_rng(3)
    U = _rand_vel(g, rng)
    v, _ = simple.project(g, tpf, _rand_vel(g, rng))
    a, _ = simple.krylov_vector(g, tpf, U, v, 50.0)
    b, _ = simple.shifted_operator(g, tpf, U, v, 50.0, 10.0)
    for c in range(3):
        np.testing.assert_allclose(a[c], b[c], atol=1e-10 * np.abs(a[c]).max())
    # a pure gradient is mapped to -sigma times itself plus a solenoidal part
    q = rng.standard_normal(g.shape_p)
    gq = [fv.gradient(g, q, c) for c in range(3)]
    y, _ = simple.shifted_operator(g, tpf, U, gq, 50.0, 10.0)
    rest = [y[c] + 10.0 * gq[c] for c in range(3)]
    assert np.abs(fv.divergence(g, rest)).max() < 1e-9 * max(np.abs(x).max() for x in rest)
