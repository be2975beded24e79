"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

Holds none of the method's arithmetic: only random draws and analytic
sample fields, produced directly in the library's storage layout.

Layout ("cell-indexed MAC", used by the C-ABI): for an nx x ny x nz grid
every field is a C-ordered float64 array of shape (nz, ny, nx); a velocity
vector is three such arrays [u | v | w] back to back (3 * nz * ny * nx
values).  u[k, j, i] is the x-velocity on the face x_i (the low face of cell
i), so u[:, :, 0] is the wall x = 0; likewise v[:, 0, :] and w[0, :, :] are
walls.  Wall entries are always zero.

Random numbers come from numpy's Philox-4x32-10 counter-based generator.
"""
import numpy as np


def _gen(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def zero_walls(vel, shape):
    nz, ny, nx = shape
    q = vel.reshape(3, nz, ny, nx)
    q[0, :, :, 0] = 0.0
    q[1, :, 0, :] = 0.0
    q[2, 0, :, :] = 0.0
    return vel


def gaussian_velocity(shape, seed):
    """Standard-normal velocity vector (walls zero), e.g. Krylov start vectors
    and right-hand sides."""
    nz, ny, nx = shape
    v = _gen(seed).standard_normal(3 * nz * ny * nx)
    return zero_walls(v, shape)


def gaussian_cells(shape, seed):
    nz, ny, nx = shape
    return _gen(seed).standard_normal(nz * ny * nx)


def map_faces(n, kind):
    """Face coordinates of the three grid maps (cosine, Eq. 5 sine, uniform)."""
    xi = np.arange(n + 1) / n
    if kind == "cosine":
        x = 0.5 * (1.0 - np.cos(np.pi * xi))
    elif kind == "sine0975":
        x = xi - 0.0975 * np.sin(2.0 * np.pi * xi)
    else:
        x = xi.copy()
    x[0], x[-1] = 0.0, 1.0
    return x


def vortex_base_flow(shape, kind="cosine", alpha=0.0):
    """A smooth lid-driven-like sample field (one recirculating vortex turned
    by the lid angle alpha plus a weak secondary flow), sampled at the face
    points; no-slip on every wall.  Used where only the structure and size of
    a base flow matter (throughput runs), not a solution of the equations."""
    nz, ny, nx = shape
    X, Y, Z = (map_faces(n, kind) for n in (nx, ny, nz))
    xc, yc, zc = ((a[1:] + a[:-1]) / 2 for a in (X, Y, Z))
    s = lambda t: np.sin(np.pi * t)
    ds = lambda t: np.pi * np.sin(2 * np.pi * t)
    ca, sa = np.cos(alpha), np.sin(alpha)

    def field(xs, ys, zs, comp):
        x, y, z = np.meshgrid(xs, ys, zs, indexing="xy")
        x, y, z = (np.transpose(a, (2, 0, 1)) for a in (x, y, z))
        psi_z = ds(z) * s(x) ** 2 * s(y) ** 2
        if comp == 0:
            return 4.0 * ca * psi_z + 0.3 * s(x) ** 2 * ds(y) * s(z) ** 2
        if comp == 1:
            return 4.0 * sa * psi_z - 0.3 * ds(x) * s(y) ** 2 * s(z) ** 2
        return -4.0 * s(z) ** 2 * (ca * ds(x) * s(y) ** 2 + sa * s(x) ** 2 * ds(y))

    u = field(X[:-1], yc, zc, 0)
    v = field(xc, Y[:-1], zc, 1)
    w = field(xc, yc, Z[:-1], 2)
    out = np.concatenate([u.ravel(), v.ravel(), w.ravel()])
    return zero_walls(out, shape)
