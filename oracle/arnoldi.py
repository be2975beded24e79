"""Implicitly restarted Arnoldi for the leading eigenvalues -- oracle.

TEST INFRASTRUCTURE ONLY.

Eq. 7: J [u; p] = lambda [u; p].  With the pressure eliminated by the
projection of Eqs. 8-9, the eigenproblem becomes A v = lambda v with
A = P L_U on divergence-free velocity fields (the pressure carries no time
derivative, so eigenvectors are velocity fields).  Section 3 runs Arnoldi
(ARPACK, Sorensen's implicitly restarted method) in regular mode for the
eigenvalues of largest real part, each Krylov vector coming from the SIMPLE
projection.

Algorithm (Sorensen 1992, exact shifts), written from its definition:
  1. v_0 = P x_0 / ||P x_0||  (x_0 is a seeded Gaussian supplied by the caller)
  2. extend the Arnoldi factorisation A V_k = V_k H_k + f e_k^T to m steps,
     orthogonalising each new vector twice (classical Gram-Schmidt, twice) in
     the W-inner product;
  3. Ritz values of H_m sorted by descending real part; the pair i is
     converged when ||f|| |e_m^T y_i| <= tol |theta_i|;
  4. otherwise apply the m - k unwanted Ritz values as shifts by implicit
     shifted QR steps on H_m (a conjugate pair by one real Francis
     double-shift step), keep k vectors and continue from step 2.

Readings: the k kept after a restart is nev + (m - nev) // 2, increased by
one when that would split a complex-conjugate pair; tolerance 1e-10.
Eigenvalues are returned sorted by descending real part, conjugate pairs
adjacent with the positive imaginary part first.  The Ritz values of the
small Hessenberg matrix use numpy.linalg.eig (a library routine used as a
step).

Pinned by (tests/test_oracle_arnoldi.py): the dense spectrum of the
projected Jacobian (oracle.dense) on grids <= 8^3; real negative spectrum of
the Stokes operator (U = 0).
"""
import numpy as np


def _sort_ritz(theta):
    """Order: descending real part; for equal real part positive imag first."""
    return sorted(range(len(theta)), key=lambda i: (-theta[i].real, -theta[i].imag))


def _keep_count(theta_sorted, k):
    """Do not split a complex-conjugate pair at position k."""
    if 0 < k < len(theta_sorted):
        a, b = theta_sorted[k - 1], theta_sorted[k]
        if abs(a.imag) > 0 and abs(a - np.conj(b)) <= 1e-12 * max(abs(a), 1.0):
            k += 1
    return k


def _house(x):
    """Householder vector v (v[0] = 1) and beta with (I - beta v v^T) x = -+||x|| e_1.

    The reflection maps x onto -sign(x_0) ||x|| e_1, so that v_0 = x_0 - (that
    value) adds two numbers of the same sign: |v_0| >= |x_0| and every
    v_i = x_i / v_0 stays below 1 in magnitude (no overflow when x_1.. are
    tiny next to x_0)."""
    x = np.asarray(x, dtype=np.float64)
    v = np.zeros_like(x)
    v[0] = 1.0
    if not np.any(x[1:]):
        return v, 0.0
    s = np.max(np.abs(x))
    xs = x / s
    norm = np.sqrt(float(xs @ xs))
    head = -norm if xs[0] >= 0 else norm          # the image -sign(x_0) ||x||
    v0 = xs[0] - head
    v[1:] = xs[1:] / v0
    beta = (head - xs[0]) / head
    return v, beta


def _francis_double_step(H, Q, c, d2):
    """One implicit double-shift QR step on the Hessenberg H for the shift
    pair c +- i sqrt(d2) (Golub & Van Loan, Algorithm 7.5.1); H <- Z^T H Z
    and Q <- Q Z, in place.  The first column of (H - mu_1)(H - mu_2) =
    (H - c)^2 + d2 is formed from h_00 - c, not from the sum and product of
    the shifts, whose expansion cancels when H is close to a multiple of
    the identity."""
    n = H.shape[0]
    a = H[0, 0] - c
    x = a * a + H[0, 1] * H[1, 0] + d2
    y = H[1, 0] * (a + H[1, 1] - c)
    z = H[1, 0] * H[2, 1] if n > 2 else 0.0
    for k in range(n - 2):
        v, beta = _house([x, y, z])
        P = np.eye(3) - beta * np.outer(v, v)
        q = max(k - 1, 0)
        H[k:k + 3, q:] = P @ H[k:k + 3, q:]
        r = min(k + 4, n)
        H[:r, k:k + 3] = H[:r, k:k + 3] @ P
        Q[:, k:k + 3] = Q[:, k:k + 3] @ P
        x = H[k + 1, k]
        y = H[k + 2, k]
        if k < n - 3:
            z = H[k + 3, k]
    v, beta = _house([x, y])
    P = np.eye(2) - beta * np.outer(v, v)
    H[n - 2:, n - 3:] = P @ H[n - 2:, n - 3:]
    H[:, n - 2:] = H[:, n - 2:] @ P
    Q[:, n - 2:] = Q[:, n - 2:] @ P


def _single_shift_step(H, Q, mu):
    """One implicit single-shift QR step (Givens bulge chase) with real shift mu."""
    n = H.shape[0]
    x, y = H[0, 0] - mu, H[1, 0]
    for k in range(n - 1):
        r = np.hypot(x, y)
        c, s = (1.0, 0.0) if r == 0.0 else (x / r, y / r)
        G = np.array([[c, -s], [s, c]])
        q = max(k - 1, 0)
        H[k:k + 2, q:] = G.T @ H[k:k + 2, q:]
        e = min(k + 3, n)
        H[:e, k:k + 2] = H[:e, k:k + 2] @ G
        Q[:, k:k + 2] = Q[:, k:k + 2] @ G
        if k < n - 2:
            x, y = H[k + 1, k], H[k + 2, k]


def arnoldi_leading(apply_A, x0, wts, nev=5, m=30, tol=1e-10, max_restarts=2000):
    """Leading nev eigenpairs of apply_A.  Returns (lam, X, info)."""
    def dot(a, b):
        return float(np.sum(wts * a * b))

    n = x0.size
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    v = np.array(x0, dtype=np.float64)
    V[0] = v / np.sqrt(dot(v, v))
    k = 0
    n_matvec = 0
    k_base = nev + (m - nev) // 2
    for restart in range(max_restarts):
        for j in range(k, m):                            # step 2
            w = apply_A(V[j])
            n_matvec += 1
            h = (V[:j + 1] * wts) @ w
            w = w - V[:j + 1].T @ h
            h2 = (V[:j + 1] * wts) @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h + h2
            beta = np.sqrt(dot(w, w))
            H[j + 1, j] = beta
            V[j + 1] = w / beta
        Hm = H[:m, :m]
        theta, Y = np.linalg.eig(Hm)                     # step 3
        order = _sort_ritz(theta)
        theta_s = theta[order]
        Y = Y[:, order]
        Y = Y / np.linalg.norm(Y, axis=0)
        fnorm = abs(H[m, m - 1])
        resid = fnorm * np.abs(Y[m - 1, :])
        scale = np.maximum(np.abs(theta_s[:nev]), np.finfo(float).eps ** (2.0 / 3.0))
        nconv = int(np.sum(resid[:nev] <= tol * scale))
        if nconv >= nev:
            X = V[:m].T @ Y[:, :nev]
            X = X / np.sqrt(np.sum(wts[:, None] * np.abs(X) ** 2, axis=0))
            for i in range(nev):                         # phase: largest entry real > 0
                big = np.argmax(np.abs(X[:, i]))
                X[:, i] *= np.conj(X[big, i]) / abs(X[big, i])
            return theta_s[:nev], X, {"restarts": restart, "matvecs": n_matvec,
                                      "resid": resid[:nev]}
        k = _keep_count(theta_s, min(k_base, m - 2))     # step 4
        shifts = list(theta_s[k:])
        Q = np.eye(m)
        Hs = Hm.copy()
        i = 0
        while i < len(shifts):
            mu = shifts[i]
            if abs(mu.imag) > 0 and i + 1 < len(shifts) and abs(shifts[i + 1] - np.conj(mu)) <= 1e-10 * abs(mu):
                _francis_double_step(Hs, Q, mu.real, mu.imag ** 2)
                i += 2
            else:
                _single_shift_step(Hs, Q, mu.real)
                i += 1
        Hs = np.triu(Hs, -1)
        Vk = Q[:, :k + 1].T @ V[:m]                      # V Q, first k+1 columns
        f = Vk[k] * Hs[k, k - 1] + V[m] * (H[m, m - 1] * Q[m - 1, k - 1])
        H[:] = 0.0
        H[:k, :k] = Hs[:k, :k]
        V[:k] = Vk[:k]
        f = f - V[:k].T @ ((V[:k] * wts) @ f)            # re-orthogonalise once
        beta = np.sqrt(dot(f, f))
        V[k] = f / beta
        H[k, k - 1] = beta
        V[k + 1:] = 0.0
    raise RuntimeError("Arnoldi did not converge")
