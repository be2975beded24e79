"""Pins of the BiCGstab(l) oracle and of Section 3's GMRES -> BiCGstab(2)
hand-off, against facts that do not come from the oracle's own code: a
direct dense solve, the textbook BiCGstab iteration (van der Vorst 1992,
written here in its p/v/s/t form) that BiCGstab(1) must reproduce step by
step, finite termination on a matrix whose minimal polynomial has degree 2,
the true residual b - A x against the recursively updated one, and the
skew-symmetric case where BiCGstab(1) stalls and BiCGstab(2) converges
(the reason Section 3 uses l = 2)."""
import numpy as np
import pytest

from oracle import fv, krylov, poisson
from oracle.grid import Grid


def _system(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    A = shift * np.eye(n) + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    w = rng.uniform(0.5, 2.0, n)
    return A, b, w


@pytest.mark.parametrize("l", [1, 2, 3])
def test_matches_direct_solve(l):
    A, b, w = _system(80, 1)
    x, mv, rel = krylov.bicgstab_l(lambda v: A @ v, b, w, l=l, tol=1e-13, max_iter=2000)
    xs = np.linalg.solve(A, b)
    assert rel <= 1e-13
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)
    assert mv % (2 * l) == 0


def _textbook_bicgstab(A, b, w, cycles):
    """van der Vorst's BiCGstab, W-inner product, shadow residual r0."""
    def dot(a, c):
        return float(np.sum(w * a * c))
    x = np.zeros_like(b)
    r = b.copy()
    rt = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho, alpha, om = 1.0, 1.0, 1.0
    xs = []
    for _ in range(cycles):
        rho1 = dot(rt, r)
        beta = (rho1 / rho) * (alpha / om)
        rho = rho1
        p = r + beta * (p - om * v)
        v = A @ p
        alpha = rho / dot(rt, v)
        s = r - alpha * v
        t = A @ s
        om = dot(t, s) / dot(t, t)
        x = x + alpha * p + om * s
        r = s - om * t
        xs.append(x.copy())
    return xs


def test_l1_reproduces_textbook_bicgstab():
    A, b, w = _system(50, 2, shift=2.0)
    ref = _textbook_bicgstab(A, b, w, 12)
    got = []
    krylov.bicgstab_l(lambda v: A @ v, b, w, l=1, tol=0.0, max_iter=24,
                      callback=lambda x, r: got.append(x.copy()))
    assert len(got) == 12
    for a, c in zip(got, ref):
        assert np.linalg.norm(a - c) <= 1e-12 * np.linalg.norm(c)


@pytest.mark.parametrize("l", [1, 2])
def test_finite_termination_minimal_polynomial_degree_two(l):
    # A = T diag(d) T^-1 with d in {1, 3}: every Krylov space has dimension
    # <= 2, so BiCG ends after two steps: one cycle of l = 2, two of l = 1
    rng = np.random.default_rng(3)
    n = 40
    T = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    d = np.where(np.arange(n) % 2 == 0, 1.0, 3.0)
    A = T @ np.diag(d) @ np.linalg.inv(T)
    b = rng.standard_normal(n)
    w = rng.uniform(0.5, 2.0, n)
    rels = []
    x, mv, rel = krylov.bicgstab_l(lambda v: A @ v, b, w, l=l, tol=0.0, max_iter=2 * l * (2 // l),
                                   callback=lambda x, r: rels.append(np.linalg.norm(b - A @ x)))
    assert mv == 4
    assert rels[-1] <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("l", [2, 3])
def test_recursive_residual_is_the_true_residual(l):
    A, b, w = _system(70, 4, shift=1.5)
    gaps = []
    krylov.bicgstab_l(lambda v: A @ v, b, w, l=l, tol=1e-12, max_iter=600,
                      callback=lambda x, r: gaps.append(np.linalg.norm((b - A @ x) - r)))
    assert len(gaps) >= 3
    assert max(gaps) <= 1e-11 * np.linalg.norm(b)


def test_l2_converges_where_l1_stalls_on_a_skew_symmetric_operator():
    # A = S + 0.01 I with S skew-symmetric: eigenvalues 0.01 +- i theta; the
    # degree-1 stabilising step of BiCGstab(1) has (A s, s) ~ 0.01 |s|^2 and
    # stalls, the degree-2 one of BiCGstab(2) handles the complex pairs
    rng = np.random.default_rng(3)
    n = 60
    rng.standard_normal((n, n))                        # same draws as a 1e-3 probe
    R = rng.standard_normal((n, n))
    A = (R - R.T) / np.sqrt(n) + 0.01 * np.eye(n)
    b = rng.standard_normal(n)
    w = np.ones(n)
    xs = np.linalg.solve(A, b)
    x2, mv2, rel2 = krylov.bicgstab_l(lambda v: A @ v, b, w, l=2, tol=1e-10, max_iter=2000)
    x1, mv1, rel1 = krylov.bicgstab_l(lambda v: A @ v, b, w, l=1, tol=1e-10, max_iter=2000)
    assert rel2 <= 1e-10 and mv2 <= 400
    assert np.linalg.norm(x2 - xs) <= 1e-8 * np.linalg.norm(xs)
    assert rel1 > 1e-6


def test_gmres_hand_off():
    # GMRES(5) saturates on this system (5 vectors per cycle are too few);
    # BiCGstab(2) then finishes from its approximation
    A, b, w = _system(120, 5, shift=1.2)
    xs = np.linalg.solve(A, b)
    x, ng, nb, rel = krylov.gmres_then_bicgstab(lambda v: A @ v, b, w, m=5, tol=1e-12,
                                                max_iter=5000, gmres_sat=0.5)
    assert ng > 0 and nb > 0
    assert rel <= 1e-12
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    # a GMRES(m) that converges in its first cycle never hands off
    x, ng, nb, rel = krylov.gmres_then_bicgstab(lambda v: A @ v, b, w, m=120, tol=1e-12,
                                                max_iter=5000, gmres_sat=0.5)
    assert nb == 0 and rel <= 1e-12


def test_zero_rhs():
    A, b, w = _system(10, 6)
    x, mv, rel = krylov.bicgstab_l(lambda v: A @ v, 0 * b, w)
    assert mv == 0 and rel == 0.0 and not x.any()


@pytest.mark.parametrize("linear", ["bicgstab", "gmres+bicgstab"])
def test_newton_steady_state_independent_of_the_linear_solver(linear, monkeypatch):
    g = Grid(8, 8, 8, "cosine")
    tpf = poisson.TPF(g)
    lid = fv.lid_velocity(0.0)
    U0, _, h0 = krylov.newton(g, tpf, 300.0, lid, tol=1e-10)
    calls = []
    inner = krylov.bicgstab_l

    def counted(*a, **k):
        calls.append(1)
        return inner(*a, **k)
    monkeypatch.setattr(krylov, "bicgstab_l", counted)
    # gmres_sat = 1e-12 hands off after every GMRES(20) cycle that does not
    # converge
    U1, _, h1 = krylov.newton(g, tpf, 300.0, lid, tol=1e-10, m=20, linear=linear,
                              gmres_sat=1e-12)
    assert len(calls) >= len(h1) - 2
    scale = max(float(np.max(np.abs(u))) for u in U0)
    assert max(float(np.max(np.abs(a - c))) for a, c in zip(U0, U1)) <= 1e-9 * scale
    assert h1[-1] < 1e-10 and len(h1) <= len(h0) + 2


def test_exact_start_needs_one_product():
    A, b, w = _system(30, 7)
    xs = np.linalg.solve(A, b)
    x, mv, rel = krylov.bicgstab_l(lambda v: A @ v, b, w, x0=xs, l=2, tol=1e-10)
    assert mv == 1 and rel <= 1e-12
    np.testing.assert_allclose(x, xs, rtol=0, atol=0)


def test_products_cap():
    # a system that needs many cycles; the cap bounds the operator products
    A, b, w = _system(150, 8, shift=0.6)
    x, mv, rel = krylov.bicgstab_l(lambda v: A @ v, b, w, l=2, tol=1e-14, max_iter=41)
    assert mv <= 41 and mv % 4 == 0
    x, ng, nb, rel = krylov.gmres_then_bicgstab(lambda v: A @ v, b, w, m=5, tol=1e-14,
                                                max_iter=60, gmres_sat=0.99)
    assert ng + nb <= 60 + 5          # GMRES counts a residual per cycle beyond its m steps
