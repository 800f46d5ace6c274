"""Staggered uniform Cartesian grid (Sec. 3, first paragraph).  TEST INFRASTRUCTURE ONLY.

Velocity nodes sit on cell faces; pressure, material properties and the extra
stress sit at cell centres.  Arrays are float64 numpy arrays of shape
``(nz, ny, nx)`` (x fastest).  The face velocity stored at index ``i`` is the one
on the +1/2 face of cell ``i`` (u at x = (i+1)dx, v at y = y0 + (j+1)dy,
w at z = (k+1)dz).

x and z are always periodic.  y is periodic or bounded by no-slip walls at
y = y0 and y = y0 + ly (the paper's channel cases, Sec. 4.1.1).  With walls the
face below cell j = 0 is the bottom wall (v = 0 there, not stored) and the stored
face ``v[:, ny-1, :]`` is the top wall, held at zero.

Ghost rules for a wall-bounded y (Reading 6):
  'c'  cell-centred scalars (B, tau, p, psi, phi): zero-gradient copy;
  'u'  u and w, centred in y: odd mirror about the wall (no slip);
  'v'  v on y-faces: zero outside the stored range (the wall faces carry v = 0).
"""

import numpy as np


class Grid:
    """Uniform staggered grid; ``walls_y`` selects no-slip walls in y."""

    def __init__(self, nx, ny, nz, lx, ly, lz, walls_y=False):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.ly, self.lz = float(lx), float(ly), float(lz)
        self.walls = bool(walls_y)
        self.dx = self.lx / self.nx
        self.dy = self.ly / self.ny
        self.dz = self.lz / self.nz
        # walls sit at y = -ly/2 and +ly/2; a periodic y starts at 0
        self.y0 = -0.5 * self.ly if self.walls else 0.0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    # coordinates of centres and faces, broadcastable to (nz, ny, nx)
    def xc(self):
        return ((np.arange(self.nx) + 0.5) * self.dx)[None, None, :]

    def yc(self):
        return (self.y0 + (np.arange(self.ny) + 0.5) * self.dy)[None, :, None]

    def zc(self):
        return ((np.arange(self.nz) + 0.5) * self.dz)[:, None, None]

    def xf(self):
        return ((np.arange(self.nx) + 1.0) * self.dx)[None, None, :]

    def yf(self):
        return (self.y0 + (np.arange(self.ny) + 1.0) * self.dy)[None, :, None]

    def zf(self):
        return ((np.arange(self.nz) + 1.0) * self.dz)[:, None, None]

    def zeros(self):
        return np.zeros(self.shape)


def _shift_y_walls(a, d, kind):
    """b[:, j, :] = a[:, j + d, :] with the wall ghost rule ``kind``."""
    ny = a.shape[1]
    j = np.arange(ny) + d
    if kind == 'c':
        return a[:, np.clip(j, 0, ny - 1), :]
    if kind == 'u':
        inside = (j >= 0) & (j < ny)
        jm = np.where(j < 0, -1 - j, np.where(j >= ny, 2 * ny - 1 - j, j))
        sign = np.where(inside, 1.0, -1.0)
        return a[:, np.clip(jm, 0, ny - 1), :] * sign[None, :, None]
    if kind == 'v':
        inside = (j >= 0) & (j < ny)
        out = a[:, np.clip(j, 0, ny - 1), :].copy()
        out[:, ~inside, :] = 0.0
        return out
    raise ValueError(kind)


def at(a, g, kind, i=0, j=0, k=0):
    """Value of field ``a`` at index offset (i, j, k) from every cell.

    ``kind`` is the field's ghost rule in a wall-bounded y ('c', 'u' or 'v');
    x and z wrap periodically, and so does y when the grid has no walls.
    """
    out = a
    if i:
        out = np.roll(out, -i, axis=2)
    if k:
        out = np.roll(out, -k, axis=0)
    if j:
        if g.walls:
            out = _shift_y_walls(out, j, kind)
        else:
            out = np.roll(out, -j, axis=1)
    return out
