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
rotations, restart), written from its definition.  BiCGstab(l) is the
algorithm of Sleijpen & Fokkema (ETNA 1, 1993): l BiCG steps that build the
powers A^j r, then a minimal-residual polynomial of degree l over them.
Section 3 runs GMRES restarted every 100 vectors until it saturates and then
BiCGstab(2) from GMRES's last approximation.  Reading of "saturates": a
restart cycle that cuts the residual W-norm by less than the factor
``gmres_sat`` (default 0.5).

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


def bicgstab_l(apply_A, b, wts, x0=None, l=2, tol=1e-12, max_iter=20000, atol=0.0,
               callback=None):
    """BiCGstab(l) in the W-inner product, shadow residual = the initial
    residual.  Stops when the (recursively updated) residual W-norm is
    <= max(tol ||b||, atol), or after max_iter matrix-vector products, or on
    a breakdown (a zero BiCG or MR denominator).  callback(x, r), if given,
    sees the iterate and its recursive residual after every cycle.
    Returns (x, matvecs, relres)."""
    def dot(a, c):
        return float(np.sum(wts * a * c))

    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.sqrt(dot(b, b))
    if bnorm == 0.0:
        return x, 0, 0.0
    stop = max(tol * bnorm, atol)
    r = np.zeros((l + 1, n))          # r[j] = A^j applied to the BiCG residual
    u = np.zeros((l + 1, n))          # u[j] = A^j applied to the BiCG direction
    r[0] = b - apply_A(x) if x0 is not None else b.copy()
    mv = 1 if x0 is not None else 0
    rt = r[0].copy()
    rho0, alpha, omega = 1.0, 0.0, 1.0
    rnorm = np.sqrt(dot(r[0], r[0]))
    while rnorm > stop and mv + 2 * l <= max_iter:
        rho0 = -omega * rho0
        # BiCG part: l steps, each raising the degree of the kept powers by one
        for j in range(l):
            rho1 = dot(r[j], rt)
            if rho0 == 0.0:
                return x, mv, rnorm / bnorm
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = apply_A(u[j])
            gam = dot(u[j + 1], rt)
            if gam == 0.0:
                return x, mv + 1, rnorm / bnorm
            alpha = rho0 / gam
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = apply_A(r[j])
            x = x + alpha * u[0]
            mv += 2
        # MR part: modified Gram-Schmidt of r[1..l], then the coefficients of
        # the degree-l polynomial that minimises the residual
        tau = np.zeros((l + 1, l + 1))
        sig = np.zeros(l + 1)
        gp = np.zeros(l + 1)           # gamma'
        for j in range(1, l + 1):
            for i in range(1, j):
                tau[i, j] = dot(r[j], r[i]) / sig[i]
                r[j] = r[j] - tau[i, j] * r[i]
            sig[j] = dot(r[j], r[j])
            if sig[j] == 0.0:
                return x, mv, rnorm / bnorm
            gp[j] = dot(r[0], r[j]) / sig[j]
        g = np.zeros(l + 2)            # gamma (g[l + 1] = 0 pads the sums)
        g[l] = gp[l]
        omega = g[l]
        for j in range(l - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, l + 1))
        gpp = np.zeros(l + 1)          # gamma''
        for j in range(1, l):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, l))
        x = x + g[1] * r[0]
        r[0] = r[0] - gp[l] * r[l]
        u[0] = u[0] - g[l] * u[l]
        for j in range(1, l):
            u[0] = u[0] - g[j] * u[j]
            x = x + gpp[j] * r[j]
            r[0] = r[0] - gp[j] * r[j]
        rnorm = np.sqrt(dot(r[0], r[0]))
        if callback is not None:
            callback(x, r[0])
    return x, mv, rnorm / bnorm


def gmres_then_bicgstab(apply_A, b, wts, m=100, tol=1e-12, max_iter=20000, atol=0.0,
                        gmres_sat=0.5, l=2):
    """Section 3's linear solver: GMRES(m) restart cycles while each cuts the
    residual W-norm by at least the factor gmres_sat; from the first cycle
    that does not (GMRES saturated), BiCGstab(l) from GMRES's last
    approximation.  max_iter caps the Krylov steps of both (Arnoldi steps
    plus residuals of GMRES, matrix-vector products of BiCGstab).
    Returns (x, gmres_matvecs, bicgstab_matvecs, relres)."""
    bnorm = np.sqrt(float(np.sum(wts * b * b)))
    if bnorm == 0.0:
        return np.zeros(b.size), 0, 0, 0.0
    stop = max(tol * bnorm, atol)
    x, its, prev = None, 0, bnorm
    while its < max_iter:
        # one restart cycle; the relres it returns is that of the true residual
        x, k, rel = gmres(apply_A, b, wts, x0=x, m=m, tol=tol, max_iter=min(m, max_iter - its),
                          atol=atol)
        its += k + 1
        if rel * bnorm <= stop:
            return x, its, 0, rel
        if rel * bnorm > gmres_sat * prev:
            break
        prev = rel * bnorm
    x, mv, rel = bicgstab_l(apply_A, b, wts, x0=x, l=l, tol=tol, max_iter=max(max_iter - its, 0),
                            atol=atol)
    return x, its, mv, rel


def steady_residual(grid, tpf, U, re, lid, forcing=None):
    """(F_m, D U, P, ||F||_inf) with P recovered by the exact projection."""
    N = fv.momentum(grid, U, re, lid, forcing)
    Fm, P = simple.project(grid, tpf, N)
    Fc = fv.divergence(grid, U)
    nrm = max(max(float(np.max(np.abs(f))) for f in Fm), float(np.max(np.abs(Fc))))
    return Fm, Fc, P, nrm


def newton(grid, tpf, re, lid, U0=None, tol=1e-10, m=100, lin_tol=1e-8,
           max_newton=30, forcing=None, max_lin_iter=20000, sigma=10.0,
           linear="gmres", gmres_sat=0.5):
    """Newton steady state (Section 3).  linear: "gmres" (restarted GMRES(m)
    only), "bicgstab" (BiCGstab(2) only) or "gmres+bicgstab" (GMRES(m) until
    it saturates, then BiCGstab(2)).  Returns (U, P, history)."""
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
        if linear == "gmres":
            du, _, _ = gmres(apply_A, fv.pack(Fm), wts, m=m, tol=lin_tol,
                             max_iter=max_lin_iter, atol=atol)
        elif linear == "bicgstab":
            du, _, _ = bicgstab_l(apply_A, fv.pack(Fm), wts, l=2, tol=lin_tol,
                                  max_iter=max_lin_iter, atol=atol)
        elif linear == "gmres+bicgstab":
            du, _, _, _ = gmres_then_bicgstab(apply_A, fv.pack(Fm), wts, m=m, tol=lin_tol,
                                              max_iter=max_lin_iter, atol=atol,
                                              gmres_sat=gmres_sat)
        else:
            raise ValueError(linear)
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
