"""Divergence-free projections onto coordinate planes and their vector
potentials (Section 4, Eqs. 11-17) -- oracle, test infrastructure.

TEST INFRASTRUCTURE ONLY.

For a velocity field v = (u, v, w) and a set of coordinate planes (a, c)
(normal direction b), the projection v_b keeps the two in-plane components,
sets the third to zero and removes the part that is not divergence-free in
the plane: v_b is the W-orthogonal projection of (in-plane part of v) onto
the fields with only those two components whose two-dimensional divergence
(Eqs. 12-14) vanishes and whose wall-normal components are zero.  On the
staggered grid this is, plane by plane (b = const), the two-dimensional
Leray projection:  solve  (L_a (+) L_c) phi = D_ac q  with Neumann walls
(phi of zero mean in each plane), then  v_b = q - G_ac phi.  The 2-D Neumann
problem is solved exactly by the 1-D eigenbases of the pressure operator
(as in poisson.TPF, without the third axis).

Vector potentials (Eqs. 15-17): v_1 = rot(0, Psi^(y), 0), v_2 =
rot(Psi^(x), 0, 0), v_3 = rot(0, 0, Psi^(z)).  The potential lives on the
corners of the plane's cells (edges along b); it vanishes on the walls and
is the running integral of the in-plane velocity across lines of the plane:
  (x, z) planes: w_1 = d Psi/dx, u_1 = -d Psi/dz;
  (y, z) planes: v_2 = d Psi/dz, w_2 = -d Psi/dy;
  (x, y) planes: u_3 = d Psi/dy, v_3 = -d Psi/dx.

Readings: the paper computes the projections "by a 2D version of the
SIMPLE-like procedure"; with the exact 2-D solve that loop ends after one
correction (as the 3-D loop does with an exact solve), which is what is
written here.  Fig. 3's projections onto planes rotated by 45 degrees are not
built (they need the field interpolated to the rotated planes).

Pinned by (tests/test_oracle_projection2d.py): zero in-plane divergence,
idempotence, W-orthogonality of the removed part, exact reconstruction of
the projection from its potential, a field already divergence-free in the
planes (built from a random potential) reproduced with its potential, and the
identity on a purely two-dimensional incompressible flow.
"""
import numpy as np

from . import fv, poisson

# planes: (in-plane axis a, in-plane axis c, normal axis b)
PLANES = {"xz": (0, 2, 1), "yz": (1, 2, 0), "xy": (0, 1, 2)}


def _apply(M, arr, d):
    a = np.moveaxis(arr, 2 - d, -1)
    a = a @ M.T
    return np.moveaxis(a, -1, 2 - d)


def _along_axis(vec, d):
    """1-D array vec laid along direction d of a [z, y, x] array (broadcastable)."""
    shape = [1, 1, 1]
    shape[2 - d] = -1
    return np.reshape(vec, shape)


def solve_2d(grid, r, a, c):
    """phi with (L_a + L_c) phi = r in every plane of constant third index
    (Neumann walls), zero mean in each plane (the null mode removed)."""
    ea, ec = poisson.AxisEigen(grid.ax[a]), poisson.AxisEigen(grid.ax[c])
    t = _apply(ea.Einv, np.asarray(r, dtype=np.float64), a)
    t = _apply(ec.Einv, t, c)
    den = _along_axis(ea.lam, a) + _along_axis(ec.lam, c)
    null = (_along_axis(np.arange(grid.ax[a].n), a) == ea.null) & \
           (_along_axis(np.arange(grid.ax[c].n), c) == ec.null)
    den = np.where(null, np.inf, den)
    t = t / den
    t = _apply(ec.E, t, c)
    return _apply(ea.E, t, a)


def divergence_2d(grid, q, a, c):
    """Two-dimensional divergence of the in-plane components a, c of q (cells)."""
    out = np.zeros(grid.shape_p)
    for d in (a, c):
        ax = grid.ax[d]
        arr = np.moveaxis(q[d], 2 - d, -1)
        out += np.moveaxis((arr[..., 1:] - arr[..., :-1]) / ax.dx, -1, 2 - d)
    return out


def project(grid, v, plane):
    """(v_b, phi): v_b the projection of v onto the planes `plane` ('xz',
    'yz' or 'xy'); the normal component of v_b is zero."""
    a, c, b = PLANES[plane]
    q = [np.zeros(grid.shape_vel(d)) for d in range(3)]
    for d in (a, c):
        q[d] = fv._zero_walls(np.array(v[d], dtype=np.float64, copy=True), d)
    phi = solve_2d(grid, divergence_2d(grid, q, a, c), a, c)
    for d in (a, c):
        q[d] = q[d] - fv.gradient(grid, phi, d)
    return q, phi


def potential(grid, vb, plane):
    """Psi^(b) of the projection vb (Eqs. 15-17) on the corners of the cells
    of the planes (a, c): a [z][y][x] array with n + 1 entries along a and c
    (the corners) and n along b (the plane index); zero on the walls.
    Running integral along a of the component c (which sits on c-faces at
    the centres along a), starting from the low a-wall."""
    a, c, b = PLANES[plane]
    n = [grid.ax[d].n for d in range(3)]
    shp = [n[2], n[1], n[0]]
    shp[2 - a] += 1
    shp[2 - c] += 1
    psi = np.zeros(shp)
    # integrate along a from its low wall: component c lives on c-faces, at
    # centres along a.  The sign follows rot: for (a, c) = (x, z), (y, z):
    # Psi_{i+1} = Psi_i + s w dx_i with s = +1 for xz, -1 for yz and for xy
    # (component v of the xy plane: Psi_{i+1} = Psi_i - v dx_i)
    sign = {"xz": 1.0, "yz": -1.0, "xy": -1.0}[plane]
    comp = np.moveaxis(vb[c], [2 - a, 2 - c], [-1, -2])     # [..., c-face, a-centre]
    out = np.moveaxis(psi, [2 - a, 2 - c], [-1, -2])        # [..., c-corner, a-corner]
    dxa = grid.ax[a].dx
    nc = grid.ax[c].n
    body = sign * comp[..., :nc, :] * dxa                    # c-faces 0..nc-1 (face nc is the wall)
    out[..., :nc, 1:] = np.cumsum(body, axis=-1)
    return np.moveaxis(out, [-1, -2], [2 - a, 2 - c])
