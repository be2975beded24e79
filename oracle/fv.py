"""Staggered (MAC) finite-volume operators -- oracle, test infrastructure.

The paper (Section 3) defers its finite-volume scheme to its reference [31];
this module writes out the reading adopted for the whole project:

* unknowns: u on x-faces, v on y-faces, w on z-faces, p at cell centres
  (wall-normal velocities are zero and are stored but are not unknowns);
* Eq. 2 is written in conservative form, d(U) = (1/Re) Lap U - div(U (x) U)
  - grad P, integrated over the momentum control volume of each face;
* diffusion: two-point gradients between neighbouring unknowns; a gradient to
  a wall uses the half-cell distance and the wall value (zero, or the lid
  velocity cos(alpha), sin(alpha) of Eq. 4 at z = 1);
* convection: the flux through a control-volume face is (transport velocity)
  x (transported velocity), each linearly interpolated (distance weighted) to
  that face; wall fluxes vanish because the wall-normal velocity is zero, so
  corner points never enter a stencil;
* continuity (Eq. 1): D U = sum_c (q_c[f+1] - q_c[f]) / dx_c.

Because every interpolation is linear, F is exactly quadratic in U and its
derivative (Eq. 6 with homogeneous boundary values, = Eq. 10 for the
momentum predictor) is computed here in closed form by ``jacvec``.

Pinned by (tests/test_oracle_fv.py): central finite differences of the
residual reproduce ``jacvec`` to round-off; second-order convergence of the
discrete solution on a manufactured solution; divergence and gradient are
negative adjoints in the volume-weighted inner products; the Stokes part is
self-adjoint; mirror symmetries of the lid-driven problem.
"""
import numpy as np


def _along(a, d):
    """View with the axis of direction d (0=x, 1=y, 2=z) moved last."""
    return np.moveaxis(a, 2 - d, -1)


def _back(a, d):
    return np.moveaxis(a, -1, 2 - d)


def _zero_walls(q, c):
    """Zero the two wall faces of component c (normal velocity at walls)."""
    a = _along(q, c)
    a[..., 0] = 0.0
    a[..., -1] = 0.0
    return q


def wall_values(c, d, lid):
    """(low, high) wall values of component c seen along tangential direction d.

    Eq. 3: zero on every wall; Eq. 4: u = cos(alpha), v = sin(alpha) at z = 1,
    which is the high wall of direction d = 2.  ``lid`` = (lid_u, lid_v)."""
    lo, hi = 0.0, 0.0
    if d == 2 and c in (0, 1):
        hi = lid[c]
    return lo, hi


def diffusion(grid, q, c, lid):
    """Lap q_c per unit control volume at the faces of component c (walls 0)."""
    out = np.zeros_like(q)
    for d in range(3):
        ax = grid.ax[d]
        a = _along(q, d)
        if d == c:
            g = (a[..., 1:] - a[..., :-1]) / ax.dx           # at cell centres
            lap = np.zeros_like(a)
            lap[..., 1:-1] = (g[..., 1:] - g[..., :-1]) / ax.dc[1:-1]
        else:
            n = ax.n
            lo, hi = wall_values(c, d, lid)
            g = np.empty(a.shape[:-1] + (n + 1,))
            g[..., 0] = (a[..., 0] - lo) / ax.dc[0]
            g[..., 1:n] = (a[..., 1:] - a[..., :-1]) / ax.dc[1:n]
            g[..., n] = (hi - a[..., n - 1]) / ax.dc[n]
            lap = (g[..., 1:] - g[..., :-1]) / ax.dx
        out += _back(lap, d)
    return _zero_walls(out, c)


def _interp_to_faces(a, ax):
    """Linear interpolation along the last axis from the n cell centres to the
    n+1 faces of ``ax``; the two wall faces are left at zero."""
    n = ax.n
    theta = 0.5 * ax.dx[:-1] / ax.dc[1:n]
    out = np.zeros(a.shape[:-1] + (n + 1,))
    out[..., 1:n] = a[..., :-1] + theta * (a[..., 1:] - a[..., :-1])
    return out


def convection(grid, a, b, c):
    """div(a (x) b_c) per unit control volume at the faces of component c.

    ``a`` (three components) is the transporting field, ``b`` the transported
    one; the residual uses a = b = U, the Jacobian a = U, b = v and a = v,
    b = U.  Wall faces of the result are 0."""
    out = np.zeros(grid.shape_vel(c))
    for d in range(3):
        axd = grid.ax[d]
        if d == c:
            A = _along(a[c], c)
            B = _along(b[c], c)
            F = (0.5 * (A[..., 1:] + A[..., :-1])) * (0.5 * (B[..., 1:] + B[..., :-1]))
            div = np.zeros_like(A)
            div[..., 1:-1] = (F[..., 1:] - F[..., :-1]) / axd.dc[1:-1]
            out += _back(div, c)
        else:
            axc = grid.ax[c]
            # transport velocity a_d: faces along d, centres along c -> c-faces
            Aint = _back(_interp_to_faces(_along(a[d], c), axc), c)
            # transported b_c: centres along d -> interior d-faces (walls: a_d = 0)
            Bint = _back(_interp_to_faces(_along(b[c], d), axd), d)
            F = _along(Aint * Bint, d)
            div = (F[..., 1:] - F[..., :-1]) / axd.dx
            out += _back(div, d)
    return _zero_walls(out, c)


def gradient(grid, p, c):
    """Component c of G p at the faces of component c (walls 0)."""
    ax = grid.ax[c]
    a = _along(p, c)
    g = np.zeros(a.shape[:-1] + (ax.n + 1,))
    g[..., 1:-1] = (a[..., 1:] - a[..., :-1]) / ax.dc[1:-1]
    return _back(g, c)


def divergence(grid, q):
    """D q at cell centres (Eq. 1)."""
    out = np.zeros(grid.shape_p)
    for c in range(3):
        ax = grid.ax[c]
        a = _along(q[c], c)
        out += _back((a[..., 1:] - a[..., :-1]) / ax.dx, c)
    return out


def lid_velocity(alpha):
    """Eq. 4: lid velocity (u, v) at z = 1 for lid angle alpha (radians)."""
    return (float(np.cos(alpha)), float(np.sin(alpha)))


def momentum(grid, U, re, lid, forcing=None):
    """N(U) = (1/Re) Lap U - div(U (x) U) (+ forcing): Eq. 2 without -grad p."""
    out = []
    for c in range(3):
        r = diffusion(grid, U[c], c, lid) / re - convection(grid, U, U, c)
        if forcing is not None:
            r = r + forcing[c]
        out.append(_zero_walls(r, c))
    return out


def residual(grid, U, P, re, lid, forcing=None):
    """Steady residual F of Eqs. 1-4: (momentum part per face, continuity per cell)."""
    N = momentum(grid, U, re, lid, forcing)
    Fm = [N[c] - gradient(grid, P, c) for c in range(3)]
    return Fm, divergence(grid, U)


def jacvec(grid, U, v, re):
    """Linearised momentum operator L_U v of Eq. 6 (homogeneous boundary values):
    (1/Re) Lap v - div(U (x) v) - div(v (x) U).  This is w of Eq. 10."""
    zero = (0.0, 0.0)
    out = []
    for c in range(3):
        r = (diffusion(grid, v[c], c, zero) / re
             - convection(grid, U, v, c) - convection(grid, v, U, c))
        out.append(_zero_walls(r, c))
    return out


# ---- inner products on the velocity space -----------------------------------

def weights(grid):
    """Momentum control-volume sizes per velocity face; 0 on wall faces (which
    are not unknowns).  The W-inner product <a, b> = sum W a b makes D and G
    negative adjoints, so the projection below is W-orthogonal."""
    return [_zero_walls(grid.face_volume(c).copy(), c) for c in range(3)]


def pack(q):
    """Three component arrays -> one flat vector (walls included)."""
    return np.concatenate([np.ravel(x) for x in q])


def unpack(grid, x):
    out, o = [], 0
    for c in range(3):
        s = grid.shape_vel(c)
        n = int(np.prod(s))
        out.append(np.array(x[o:o + n]).reshape(s))
        o += n
    return out
