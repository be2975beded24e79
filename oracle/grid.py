"""Stretched staggered grid of Section 3 (Eq. 5) -- oracle, test infrastructure.

Face coordinates x_i = s(i/N), i = 0..N, with three maps:

* ``"sine0975"`` -- Eq. 5: s(xi) = xi - 0.0975 sin(2 pi xi).
* ``"cosine"``   -- s(xi) = (1 - cos(pi xi)) / 2, the stretching used by the
                    benchmark configurations of this project.
* ``"uniform"``  -- s(xi) = xi.

Per axis the finite-volume metrics are
  dx[m]  = x[m+1] - x[m]             (cell widths, m = 0..N-1),
  xc[m]  = (x[m] + x[m+1]) / 2       (cell centres),
  dc[f]  = xc[f] - xc[f-1]           (centre spacing at interior face f),
  dc[0]  = dx[0] / 2, dc[N] = dx[N-1] / 2   (half cell to the wall).

Pinned by: the Eq. 5 step sizes quoted in Section 3 (smallest step
~0.387/N, largest ~1.387/N) and by closed-form values of the cosine map.
"""
import numpy as np

MAPS = ("sine0975", "cosine", "uniform")


def faces(n, kind):
    """Face coordinates x_0..x_n of one axis (Section 3, Eq. 5)."""
    xi = np.arange(n + 1, dtype=np.float64) / n
    if kind == "sine0975":
        x = xi - 0.0975 * np.sin(2.0 * np.pi * xi)
    elif kind == "cosine":
        x = 0.5 * (1.0 - np.cos(np.pi * xi))
    elif kind == "uniform":
        x = xi.copy()
    else:
        raise ValueError(f"unknown grid map {kind!r}")
    x[0] = 0.0
    x[-1] = 1.0
    return x


class Axis:
    """Metrics of one axis with n cells."""

    def __init__(self, n, kind):
        if n < 2:
            raise ValueError("an axis needs at least 2 cells")
        self.n = n
        self.x = faces(n, kind)
        self.dx = np.diff(self.x)
        self.xc = 0.5 * (self.x[:-1] + self.x[1:])
        dc = np.empty(n + 1)
        dc[0] = 0.5 * self.dx[0]
        dc[1:n] = np.diff(self.xc)
        dc[n] = 0.5 * self.dx[n - 1]
        self.dc = dc


class Grid:
    """N_x x N_y x N_z staggered grid on the unit cube.

    Array index order everywhere in the oracle is [k, j, i] = [z, y, x].
    Velocity components include their wall faces:
      u: (nz, ny, nx+1), v: (nz, ny+1, nx), w: (nz+1, ny, nx), p: (nz, ny, nx).
    """

    def __init__(self, nx, ny, nz, kind="cosine"):
        self.kind = kind
        self.ax = (Axis(nx, kind), Axis(ny, kind), Axis(nz, kind))
        self.nx, self.ny, self.nz = nx, ny, nz

    @property
    def shape_p(self):
        return (self.nz, self.ny, self.nx)

    def shape_vel(self, c):
        """Array shape of velocity component c (0=u, 1=v, 2=w), walls included."""
        s = [self.nz, self.ny, self.nx]
        s[2 - c] += 1
        return tuple(s)

    def zeros_vel(self):
        return [np.zeros(self.shape_vel(c)) for c in range(3)]

    def cell_volume(self):
        X, Y, Z = self.ax
        return Z.dx[:, None, None] * Y.dx[None, :, None] * X.dx[None, None, :]

    def face_volume(self, c):
        """Control-volume size of the component-c momentum cell at every face
        (walls get the half-cell volume; they are not unknowns)."""
        X, Y, Z = self.ax
        lx = X.dc if c == 0 else X.dx
        ly = Y.dc if c == 1 else Y.dx
        lz = Z.dc if c == 2 else Z.dx
        return lz[:, None, None] * ly[None, :, None] * lx[None, None, :]
