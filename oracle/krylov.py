"""GMRES(m) and the Newton method of Section 3 -- oracle, test infrastructure.

Newton (Section 3, steps 1-4): from a guess (U, P) compute the residual F of
Eqs. 1-4; stop when ||F|| < eps; otherwise solve J [u; p] = F and update
U -= u, P -= p.

Readings: the pressure is eliminated by the projection, i.e. P(U) is the
zero-mean solution of D G P = D N(U), so the momentum residual is the
projected one, F_m = N(U) - G P(U); the continuity residual is D U, which
stays zero because every correction is divergence-free.  ||F|| is the max
norm over both parts.  The correction u solves P L_U u = F_m on the
divergence-free subspace by restarted GMRES(m) whose Krylov vectors are the
SIMPLE projections of Eq. 8 (Section 3: GMRES restarted every 100 vectors),
applied in the shifted form of ``simple.shifted_operator`` so that the
gradient complement, which the right-hand side never excites, is not a
null space of the operator.
Inner products are the control-volume weighted ones (``fv.weights``).

GMRES is the textbook algorithm (Arnoldi with modified Gram-Schmidt, Givens
rotations, restart), written from its definition.

Pinned by: the manufactured-solution test (Newton reaches the discrete
solution, whose error then shows second-order convergence); quadratic
decrease of ||F||; symmetry of the computed steady states.
"""
import numpy as np

from . import fv, simple


def gmres(apply_A, b, wts, x0=None, m=100, tol=1e-12, max_iter=20000, atol=0.0):
    """Restarted GMRES(m) in the W-inner product; stops when the residual
    W-norm is <= max(tol ||b||, atol).  Returns (x, iters, relres)."""
    def dot(a, c):
        return float(np.sum(wts * a * c))

    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.sqrt(dot(b, b))
    if bnorm == 0.0:
        return x, 0, 0.0
    stop = max(tol * bnorm, atol)
    its = 0
    x_is_zero = x0 is None
    while True:
        r = b.copy() if x_is_zero else b - apply_A(x)
        x_is_zero = False
        beta = np.sqrt(dot(r, r))
        if beta <= stop or its >= max_iter:
            return x, its, beta / bnorm
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = apply_A(V[j])
            for i in range(j + 1):                     # modified Gram-Schmidt
                H[i, j] = dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.sqrt(dot(w, w))
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                         # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) <= stop or its >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + V[:j_done].T @ y


def steady_residual(grid, tpf, U, re, lid, forcing=None):
    """(F_m, D U, P, ||F||_inf) with P recovered by the exact projection."""
    N = fv.momentum(grid, U, re, lid, forcing)
    Fm, P = simple.project(grid, tpf, N)
    Fc = fv.divergence(grid, U)
    nrm = max(max(float(np.max(np.abs(f))) for f in Fm), float(np.max(np.abs(Fc))))
    return Fm, Fc, P, nrm


def newton(grid, tpf, re, lid, U0=None, tol=1e-10, m=100, lin_tol=1e-8,
           max_newton=30, forcing=None, max_lin_iter=20000, sigma=10.0):
    """Newton steady state (Section 3).  Returns (U, P, history)."""
    U = grid.zeros_vel() if U0 is None else [np.array(x, dtype=np.float64, copy=True) for x in U0]
    wts = fv.pack(fv.weights(grid))
    # W-norm floor that still guarantees a max-norm residual well below tol
    atol = 1e-3 * tol * float(np.sqrt(np.min(wts[wts > 0])))
    hist = []
    for _ in range(max_newton + 1):
        # continuity part of the Newton correction: J [u; p] = F with
        # D u = D U is solved by the gradient part of u, i.e. U is projected
        # (removes the divergence that round-off accumulates in U)
        U, _ = simple.project(grid, tpf, U)
        Fm, Fc, P, nrm = steady_residual(grid, tpf, U, re, lid, forcing)
        hist.append(nrm)
        if nrm < tol:
            return U, P, hist
        if len(hist) > max_newton:
            break

        def apply_A(x, U=U):
            v, _ = simple.shifted_operator(grid, tpf, U, fv.unpack(grid, x), re, sigma)
            return fv.pack(v)

        # the correction only has to be accurate to well below the Newton
        # tolerance; asking for more stalls GMRES at round-off level
        du, _, _ = gmres(apply_A, fv.pack(Fm), wts, m=m, tol=lin_tol,
                         max_iter=max_lin_iter, atol=atol)
        du = fv.unpack(grid, du)
        U = [U[c] - du[c] for c in range(3)]
    raise RuntimeError(f"Newton did not converge: {hist}")


def newton_continuation(grid, tpf, re_path, lid, tol=1e-10, m=100, lin_tol=1e-8):
    """Newton along a sequence of Re values, each warm-started from the last
    (from rest at the first one)."""
    U = None
    allhist = []
    for re in re_path:
        U, P, hist = newton(grid, tpf, re, lid, U0=U, tol=tol, m=m, lin_tol=lin_tol)
        allhist.append((re, hist))
    return U, P, allhist
