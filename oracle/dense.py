"""Brute-force dense spectrum of the linearised problem -- oracle.

TEST INFRASTRUCTURE ONLY; small grids (<= 8^3) only.

Eq. 7 with the continuity constraint: L_U v - G q = lambda v, D v = 0.  Two
independent dense constructions of the same finite spectrum:

* ``reduced_spectrum``: a W-orthonormal basis Z of the null space of D
  (SVD of D W^{-1/2}, numpy), then eig(Z^T W L_U Z).  Because the projection
  is W-orthogonal, Z^T W P L_U Z = Z^T W L_U Z.
* ``pencil_spectrum``: the finite eigenvalues of the saddle-point pencil
  ([[L, -G], [D, 0]], diag(I, 0)) by the QZ algorithm (scipy.linalg.eig),
  after removing the constant-pressure null mode (one pressure unknown and
  one dependent continuity row dropped).

The matrix of L_U is assembled column by column from ``fv.jacvec`` applied
to unit vectors.  Parity of the two constructions with each other is the
pin of this module.
"""
import numpy as np

from . import fv


def interior_index(grid):
    """Flat indices (in fv.pack order) of the velocity unknowns (no wall faces)."""
    wts = fv.pack(fv.weights(grid))
    return np.nonzero(wts > 0)[0], wts


def assemble_L(grid, U, re):
    idx, _ = interior_index(grid)
    n_all = fv.pack(grid.zeros_vel()).size
    L = np.zeros((idx.size, idx.size))
    e = np.zeros(n_all)
    for col, g in enumerate(idx):
        e[g] = 1.0
        L[:, col] = fv.pack(fv.jacvec(grid, U, fv.unpack(grid, e), re))[idx]
        e[g] = 0.0
    return L


def assemble_D(grid):
    idx, _ = interior_index(grid)
    n_all = fv.pack(grid.zeros_vel()).size
    D = np.zeros((int(np.prod(grid.shape_p)), idx.size))
    e = np.zeros(n_all)
    for col, g in enumerate(idx):
        e[g] = 1.0
        D[:, col] = fv.divergence(grid, fv.unpack(grid, e)).ravel()
        e[g] = 0.0
    return D


def reduced_spectrum(grid, U, re, L=None):
    idx, wts = interior_index(grid)
    w = wts[idx]
    if L is None:
        L = assemble_L(grid, U, re)
    D = assemble_D(grid)
    s = np.sqrt(w)
    M = D / s[None, :]
    _, sv, Vt = np.linalg.svd(M)
    rank = int(np.sum(sv > sv[0] * 1e-12))
    Zp = Vt[rank:].T                               # orthonormal null space of M
    Ared = Zp.T @ (s[:, None] * L / s[None, :]) @ Zp
    lam = np.linalg.eigvals(Ared)
    return lam[np.lexsort((-lam.imag, -lam.real))]


def pencil_spectrum(grid, U, re, L=None):
    import scipy.linalg as sla
    idx, _ = interior_index(grid)
    if L is None:
        L = assemble_L(grid, U, re)
    D = assemble_D(grid)
    # G = -W_v^{-1} D^T W_p; build it directly from fv.gradient instead
    npc = D.shape[0]
    n_all = fv.pack(grid.zeros_vel()).size
    G = np.zeros((idx.size, npc))
    e = np.zeros(npc)
    for col in range(npc):
        e[col] = 1.0
        G[:, col] = fv.pack([fv.gradient(grid, e.reshape(grid.shape_p), c) for c in range(3)])[idx]
        e[col] = 0.0
    nv = idx.size
    keep_p = np.arange(1, npc)                     # drop the constant-pressure mode
    A = np.zeros((nv + npc - 1, nv + npc - 1))
    A[:nv, :nv] = L
    A[:nv, nv:] = -G[:, keep_p]
    A[nv:, :nv] = D[1:, :]
    B = np.zeros_like(A)
    B[:nv, :nv] = np.eye(nv)
    alpha, beta = sla.eig(A, B, right=False, homogeneous_eigvals=True)
    finite = np.abs(beta) > 1e-10 * np.abs(alpha).max()
    lam = alpha[finite] / beta[finite]
    assert n_all >= nv
    return lam[np.lexsort((-lam.imag, -lam.real))]
