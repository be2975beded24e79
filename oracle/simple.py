"""SIMPLE-like evaluation of Krylov vectors (Section 3, Eqs. 8-10) -- oracle.

TEST INFRASTRUCTURE ONLY.

The next Krylov vector (v', p') must satisfy Eq. 8,
  v' = -grad p' + (1/Re) Lap v - (U.grad) v - (v.grad) U,
together with Eq. 9 (div v' = 0 and the homogeneous boundary conditions).
Section 3 reads this as the projection of w (Eq. 10) onto divergence-free
fields and computes it by the loop

  v' = w, p' = 0; repeat { solve Lap phi = div v' (Neumann);
                           v' -= grad phi; p' += phi;
                           restore boundary values of v' } until ||phi|| < eps.

Readings used here:
* on the staggered grid the wall-normal velocities are not unknowns and the
  tangential boundary values live inside the stencils, so the "restore
  boundary conditions" step changes nothing; the loop repeats only when the
  Poisson solve of step 1 is inexact (defect correction);
* ||phi|| is the max norm, and the stop test is relative to the first
  correction: ||phi_k|| <= eps * ||phi_1||;
* an optional under-relaxation factor omega scales each correction
  (omega = 1 is the paper's algorithm; the fixed point does not depend on it).

``krylov_vector`` is the plain definition (one exact projection);
``simple_loop`` runs the paper's loop with any Poisson solver, so that a test
can show an inexact solver reaching the same fixed point.
"""
import numpy as np

from . import fv


def project(grid, tpf, w):
    """Exact W-orthogonal projection: (v, p) with v = w - G p, D v = 0."""
    r = fv.divergence(grid, w)
    phi = tpf.solve(r)
    v = [w[c] - fv.gradient(grid, phi, c) for c in range(3)]
    return v, phi


def krylov_vector(grid, tpf, U, v, re):
    """Eqs. 8-9 by definition: (P L_U v, p) with one exact projection."""
    w = fv.jacvec(grid, U, v, re)
    return project(grid, tpf, w)


def shifted_operator(grid, tpf, U, v, re, sigma):
    """A_sigma v = P (L_U v + sigma v) - sigma v.

    On divergence-free v this equals the Krylov vector of Eqs. 8-9
    (P v = v).  On the gradient complement it acts as -sigma, so the
    non-solenoidal directions that round-off feeds into an Arnoldi or GMRES
    basis get the eigenvalue -sigma instead of 0 and are never "leading"
    (in regular-mode Arnoldi a zero eigenvalue outranks the negative real
    parts of a stable flow and is amplified by every restart).  One
    projection per application, as for the plain Krylov vector."""
    w = fv.jacvec(grid, U, v, re)
    w = [w[c] + sigma * v[c] for c in range(3)]
    y, p = project(grid, tpf, w)
    return [y[c] - sigma * v[c] for c in range(3)], p


def simple_loop(grid, w, poisson_solve, eps=1e-8, max_pass=200, omega=1.0):
    """The three-step loop of Section 3 starting from w.

    Returns (v, p, phi_norms).  ``poisson_solve(r)`` returns an (approximate)
    solution of D G phi = r."""
    v = [np.array(x, dtype=np.float64, copy=True) for x in w]
    p = np.zeros(grid.shape_p)
    norms = []
    for _ in range(max_pass):
        r = fv.divergence(grid, v)                         # step 1
        phi = omega * poisson_solve(r)
        for c in range(3):                                 # step 2
            v[c] -= fv.gradient(grid, phi, c)
        p += phi
        # step 3: boundary values are part of the stencils on this grid (no-op)
        nrm = float(np.max(np.abs(phi)))
        norms.append(nrm)
        if nrm == 0.0 or nrm <= eps * norms[0]:
            return v, p, norms
    raise RuntimeError(f"SIMPLE loop did not converge in {max_pass} passes: {norms[-3:]}")
