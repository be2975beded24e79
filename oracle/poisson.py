"""Exact Neumann pressure-correction solve -- oracle, test infrastructure.

Step 1 of the SIMPLE-like algorithm of Section 3 solves Lap phi = div v with
d phi / dn = 0.  Discretely the operator is D G (divergence of the gradient),
which on a tensor-product grid is separable:

  D G = L_x (x) I (x) I + I (x) L_y (x) I + I (x) I (x) L_z,
  (L phi)_m = [ (phi_{m+1}-phi_m)/dc_{m+1} - (phi_m-phi_{m-1})/dc_m ] / dx_m,

with the wall fluxes (m = 0 low side, m = n-1 high side) equal to zero.
Section 3 solves it "analytically" by eigen-decomposition of the 1-D
second-derivative operators (TPF, tensor-product factorisation).  Here
L = dx^{-1} T with T symmetric, so S = dx^{-1/2} T dx^{-1/2} = Q Lam Q^T and
L = E Lam E^{-1}, E = dx^{-1/2} Q, E^{-1} = Q^T dx^{1/2}.  The rhs is
transformed along x, y, z, divided by lam_x + lam_y + lam_z, the single
null mode (the constant) is set to zero (phi has zero volume mean), and the
result is transformed back.

The 1-D symmetric eigenproblems use numpy.linalg.eigh (a library routine
used as one step).

Pinned by (tests/test_oracle_poisson.py): the closed-form eigenvalues
-(2/h sin(k pi / 2n))^2 of the uniform Neumann operator; D G phi = r to
round-off on random compatible right-hand sides; zero volume mean.
"""
import numpy as np


def neumann_matrix(ax):
    """(L, T): the 1-D Neumann operator L = dx^{-1} T and its symmetric T."""
    n = ax.n
    T = np.zeros((n, n))
    for f in range(1, n):           # interior face f between cells f-1 and f
        g = 1.0 / ax.dc[f]
        T[f - 1, f - 1] -= g
        T[f, f] -= g
        T[f - 1, f] += g
        T[f, f - 1] += g
    return T / ax.dx[:, None], T


class AxisEigen:
    """Eigen-decomposition L = E diag(lam) E^{-1} of one 1-D Neumann operator."""

    def __init__(self, ax):
        _, T = neumann_matrix(ax)
        s = np.sqrt(ax.dx)
        S = T / s[:, None] / s[None, :]
        lam, Q = np.linalg.eigh(S)
        self.lam = lam
        self.E = Q / s[:, None]
        self.Einv = Q.T * s[None, :]
        self.null = int(np.argmax(lam))     # the zero eigenvalue (constant mode)


def _apply(M, a, d):
    """Apply matrix M along direction d (0=x, 1=y, 2=z) of a [z, y, x] array."""
    a = np.moveaxis(a, 2 - d, -1)
    a = a @ M.T
    return np.moveaxis(a, -1, 2 - d)


class TPF:
    """Exact solver of D G phi = r (Neumann, zero-mean phi) on a Grid."""

    def __init__(self, grid):
        self.grid = grid
        self.eig = [AxisEigen(grid.ax[d]) for d in range(3)]
        ex, ey, ez = self.eig
        den = ez.lam[:, None, None] + ey.lam[None, :, None] + ex.lam[None, None, :]
        den[ez.null, ey.null, ex.null] = np.inf
        self.inv_den = 1.0 / den            # null mode -> 0

    def solve(self, r):
        a = np.asarray(r, dtype=np.float64)
        for d in range(3):
            a = _apply(self.eig[d].Einv, a, d)
        a = a * self.inv_den
        for d in range(3):
            a = _apply(self.eig[d].E, a, d)
        return a


def apply_DG(grid, phi):
    """D G phi written out directly from the 1-D operators (for checks)."""
    out = np.zeros_like(phi)
    for d in range(3):
        L, _ = neumann_matrix(grid.ax[d])
        out += _apply(L, phi, d)
    return out
