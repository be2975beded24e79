"""Pins of the oracle finite-volume operators (Section 3, Eqs. 1-4, 6, 10)."""
import numpy as np
import pytest

from oracle import fv, grid as G, poisson, simple, krylov
import mms


def _rand_vel(g, rng):
    return [fv._zero_walls(rng.standard_normal(g.shape_vel(c)), c) for c in range(3)]


@pytest.mark.parametrize("kind", G.MAPS)
@pytest.mark.parametrize("h", [1.0, 1e-3])
def test_jacvec_equals_central_difference_of_residual(kind, h):
    # F is quadratic in U, so the central difference is exact for any h; the
    # analytic J.v must agree with it to round-off (<< 1e-6)
    g = G.Grid(5, 6, 7, kind)
    rng = np.random.default_rng(0)
    U, v = _rand_vel(g, rng), _rand_vel(g, rng)
    P = rng.standard_normal(g.shape_p)
    lid, re = fv.lid_velocity(0.3), 137.0
    Jv = fv.jacvec(g, U, v, re)
    Fp, _ = fv.residual(g, [U[c] + h * v[c] for c in range(3)], P, re, lid)
    Fm, _ = fv.residual(g, [U[c] - h * v[c] for c in range(3)], P, re, lid)
    scale = max(np.abs(Jv[c]).max() for c in range(3))
    for c in range(3):
        np.testing.assert_allclose((Fp[c] - Fm[c]) / (2 * h), Jv[c], atol=1e-10 * scale / min(h, 1.0) * 1e-3)


def test_divergence_gradient_adjoint():
    g = G.Grid(6, 5, 4, "cosine")
    rng = np.random.default_rng(1)
    U = _rand_vel(g, rng)
    q = rng.standard_normal(g.shape_p)
    W = fv.weights(g)
    lhs = (fv.divergence(g, U) * q * g.cell_volume()).sum()
    rhs = -sum((W[c] * U[c] * fv.gradient(g, q, c)).sum() for c in range(3))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_stokes_operator_self_adjoint_negative():
    # U = 0: L_0 = (1/Re) Lap is W-symmetric and negative definite
    g = G.Grid(5, 4, 6, "sine0975")
    rng = np.random.default_rng(2)
    a, b = _rand_vel(g, rng), _rand_vel(g, rng)
    Z = g.zeros_vel()
    W = fv.weights(g)
    La, Lb = fv.jacvec(g, Z, a, 3.0), fv.jacvec(g, Z, b, 3.0)
    ab = sum((W[c] * La[c] * b[c]).sum() for c in range(3))
    ba = sum((W[c] * a[c] * Lb[c]).sum() for c in range(3))
    np.testing.assert_allclose(ab, ba, rtol=1e-12)
    assert sum((W[c] * La[c] * a[c]).sum() for c in range(3)) < 0


def test_lid_enters_only_tangential_diffusion():
    # Eq. 4: the lid value appears in the z-diffusion of u and v next to z = 1
    g = G.Grid(4, 4, 5, "cosine")
    Z = g.zeros_vel()
    P = np.zeros(g.shape_p)
    Fm, Fc = fv.residual(g, Z, P, 2.0, (1.0, 0.0))
    assert np.all(Fc == 0)
    nz_u = np.argwhere(Fm[0] != 0)
    assert set(nz_u[:, 0]) == {g.nz - 1}
    expect = 1.0 / 2.0 / g.ax[2].dc[-1] / g.ax[2].dx[-1]
    np.testing.assert_allclose(Fm[0][-1, :, 1:-1], expect, rtol=1e-14)
    assert np.all(Fm[1] == 0) and np.all(Fm[2] == 0)


def test_convection_conserves_momentum_uniform():
    # conservative form on a uniform grid: the volume integral of div(a b) over
    # all u-faces telescopes to the wall fluxes, which vanish (no-slip)
    g = G.Grid(6, 6, 6, "uniform")
    rng = np.random.default_rng(4)
    a, b = _rand_vel(g, rng), _rand_vel(g, rng)
    for c in range(3):
        # boundary faces of the c-CV chain along c: flux at half cells is nonzero,
        # so compare against the explicit wall-centre fluxes
        C = fv.convection(g, a, b, c)
        W = fv.face_volume_sum = None
        tot = (fv.weights(g)[c] * C).sum()
        A = np.moveaxis(a[c], 2 - c, -1)
        B = np.moveaxis(b[c], 2 - c, -1)
        F0 = 0.5 * (A[..., 0] + A[..., 1]) * 0.5 * (B[..., 0] + B[..., 1])
        F1 = 0.5 * (A[..., -1] + A[..., -2]) * 0.5 * (B[..., -1] + B[..., -2])
        area = 1.0 / 36.0
        np.testing.assert_allclose(tot, area * (F1.sum() - F0.sum()), atol=1e-12)


def test_projection_properties():
    g = G.Grid(6, 7, 5, "cosine")
    tpf = poisson.TPF(g)
    rng = np.random.default_rng(5)
    w = _rand_vel(g, rng)
    v, p = simple.project(g, tpf, w)
    assert np.abs(fv.divergence(g, v)).max() < 1e-12 * max(np.abs(x).max() for x in w) / g.ax[0].dx.min()
    v2, p2 = simple.project(g, tpf, v)                     # idempotent
    for c in range(3):
        np.testing.assert_allclose(v2[c], v[c], atol=1e-12)
    W = fv.weights(g)                                      # W-orthogonal
    ip = sum((W[c] * v[c] * (w[c] - v[c])).sum() for c in range(3))
    nn = sum((W[c] * w[c] * w[c]).sum() for c in range(3))
    assert abs(ip) < 1e-13 * nn


@pytest.mark.parametrize("kind", ["uniform", "sine0975", "cosine"])
def test_second_order_convergence_manufactured(kind):
    # discrete solution error O(h^2) on a manufactured steady solution
    # (Newton from rest, Re = 10, all walls at rest)
    pytest.importorskip("sympy")
    re = 10.0
    Uf, Pf, ff = mms.build(re)
    errs = []
    for n in (8, 16):
        g = G.Grid(n, n, n, kind)
        f = [fv._zero_walls(x, c) for c, x in enumerate(mms.sample(g, ff))]
        Ue = mms.sample(g, Uf)
        U, P, hist = krylov.newton(g, poisson.TPF(g), re, (0.0, 0.0), forcing=f, tol=1e-10, lin_tol=1e-8)
        errs.append(max(np.abs(U[c] - Ue[c]).max() for c in range(3)))
    assert 3.4 < errs[0] / errs[1] < 4.6, errs


def test_newton_quadratic_and_symmetric_alpha0():
    # alpha = 0: mirror symmetry about y = 1/2 (v odd, u and w even)
    g = G.Grid(6, 6, 6, "cosine")
    U, P, hist = krylov.newton(g, poisson.TPF(g), 100.0, fv.lid_velocity(0.0))
    assert hist[-1] < 1e-10
    assert any(hist[i + 1] < 10 * hist[i] ** 2 for i in range(len(hist) - 1))
    np.testing.assert_allclose(U[0], U[0][:, ::-1, :], atol=1e-11)
    np.testing.assert_allclose(U[2], U[2][:, ::-1, :], atol=1e-11)
    np.testing.assert_allclose(U[1], -U[1][:, ::-1, :], atol=1e-11)


def test_newton_symmetric_alpha45():
    # alpha = 45 deg: invariant under the swap x <-> y with u <-> v
    g = G.Grid(6, 6, 6, "cosine")
    U, P, hist = krylov.newton(g, poisson.TPF(g), 100.0, fv.lid_velocity(np.pi / 4))
    np.testing.assert_allclose(U[0], np.swapaxes(U[1], 1, 2), atol=1e-11)
    np.testing.assert_allclose(U[2], np.swapaxes(U[2], 1, 2), atol=1e-11)
