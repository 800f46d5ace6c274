"""Momentum right-hand side of Eqs. NS, ru and NS-num1 (Secs. 2, 3.2.2, 3.3.1).
TEST INFRASTRUCTURE ONLY.

Second-order central differences on the staggered grid (Sec. 3):
  * div(uu) at each face from products at cell centres (normal part) and at cell
    edges (cross part, each factor the average of its two neighbours);
  * the viscous term div[mu_s (grad u + grad u^T)]; with a uniform mu_s it is taken
    as mu_s times the 7-point Laplacian (Reading 3b: the transpose part is
    mu_s grad(div u), zero for the projected velocity it acts on); with a variable
    mu_s (two-phase mixture, Sec. 3.2.1) the full form is used;
  * div(tau) at faces from centre tau, the off-diagonal parts through edge values
    that are 4-point averages of the centre values (Reading 5);
  * grad p at faces from the two neighbouring centres.

Fields with walls: the top y-face v[:, ny-1, :] is the wall and stays zero.
"""

import numpy as np

from .grid import at
from .models import comp_index


def advection(U, V, W, g):
    """div(uu) at the u, v and w faces."""
    dx, dy, dz = g.dx, g.dy, g.dz

    def avg(a, b):
        return 0.5 * (a + b)

    # --- x-face (i+1/2, j, k)
    uu_hi = avg(U, at(U, g, 'u', i=1)) ** 2          # centre i+1
    uu_lo = avg(at(U, g, 'u', i=-1), U) ** 2         # centre i
    uv_hi = avg(U, at(U, g, 'u', j=1)) * avg(V, at(V, g, 'v', i=1))               # edge (i+1/2, j+1/2)
    uv_lo = (avg(at(U, g, 'u', j=-1), U)
             * avg(at(V, g, 'v', j=-1), at(V, g, 'v', i=1, j=-1)))                # edge (i+1/2, j-1/2)
    uw_hi = avg(U, at(U, g, 'u', k=1)) * avg(W, at(W, g, 'u', i=1))               # edge (i+1/2, k+1/2)
    uw_lo = avg(at(U, g, 'u', k=-1), U) * avg(at(W, g, 'u', k=-1), at(W, g, 'u', i=1, k=-1))
    Ax = (uu_hi - uu_lo) / dx + (uv_hi - uv_lo) / dy + (uw_hi - uw_lo) / dz

    # --- y-face (i, j+1/2, k)
    vu_hi = avg(U, at(U, g, 'u', j=1)) * avg(V, at(V, g, 'v', i=1))               # edge (i+1/2, j+1/2)
    vu_lo = (avg(at(U, g, 'u', i=-1), at(U, g, 'u', i=-1, j=1))
             * avg(at(V, g, 'v', i=-1), V))                                        # edge (i-1/2, j+1/2)
    vv_hi = avg(V, at(V, g, 'v', j=1)) ** 2          # centre j+1
    vv_lo = avg(at(V, g, 'v', j=-1), V) ** 2         # centre j
    vw_hi = avg(V, at(V, g, 'v', k=1)) * avg(W, at(W, g, 'u', j=1))               # edge (j+1/2, k+1/2)
    vw_lo = (avg(at(V, g, 'v', k=-1), V)
             * avg(at(W, g, 'u', k=-1), at(W, g, 'u', j=1, k=-1)))                 # edge (j+1/2, k-1/2)
    Ay = (vu_hi - vu_lo) / dx + (vv_hi - vv_lo) / dy + (vw_hi - vw_lo) / dz

    # --- z-face (i, j, k+1/2)
    wu_hi = avg(U, at(U, g, 'u', k=1)) * avg(W, at(W, g, 'u', i=1))               # edge (i+1/2, k+1/2)
    wu_lo = (avg(at(U, g, 'u', i=-1), at(U, g, 'u', i=-1, k=1))
             * avg(at(W, g, 'u', i=-1), W))                                        # edge (i-1/2, k+1/2)
    wv_hi = avg(V, at(V, g, 'v', k=1)) * avg(W, at(W, g, 'u', j=1))               # edge (j+1/2, k+1/2)
    wv_lo = (avg(at(V, g, 'v', j=-1), at(V, g, 'v', j=-1, k=1))
             * avg(at(W, g, 'u', j=-1), W))                                        # edge (j-1/2, k+1/2)
    ww_hi = avg(W, at(W, g, 'u', k=1)) ** 2
    ww_lo = avg(at(W, g, 'u', k=-1), W) ** 2
    Az = (wu_hi - wu_lo) / dx + (wv_hi - wv_lo) / dy + (ww_hi - ww_lo) / dz
    return Ax, Ay, Az


def laplacian(F, g, kind):
    """7-point Laplacian of a face (or centre) field with its ghost rule."""
    return ((at(F, g, kind, i=1) - 2.0 * F + at(F, g, kind, i=-1)) / g.dx ** 2
            + (at(F, g, kind, j=1) - 2.0 * F + at(F, g, kind, j=-1)) / g.dy ** 2
            + (at(F, g, kind, k=1) - 2.0 * F + at(F, g, kind, k=-1)) / g.dz ** 2)


def viscous(U, V, W, g, mu_s):
    """div[mu_s (grad u + grad u^T)] at the faces.

    Uniform mu_s: mu_s * Laplacian (Reading 3b).  Array mu_s (cell centres):
    the full form -- normal stresses at centres, shear stresses at edges with
    the edge viscosity the 4-point average of the surrounding centre values."""
    if np.ndim(mu_s) == 0:
        return (mu_s * laplacian(U, g, 'u'), mu_s * laplacian(V, g, 'v'),
                mu_s * laplacian(W, g, 'u'))
    dx, dy, dz = g.dx, g.dy, g.dz
    mu = mu_s

    def mu_edge(**offs):
        # mu averaged over the 4 centres around an edge: offsets (0 or a) x (0 or b)
        return _avg4(mu, g, **offs)

    # normal viscous stresses at centres
    sxx = 2.0 * mu * (U - at(U, g, 'u', i=-1)) / dx
    syy = 2.0 * mu * (V - at(V, g, 'v', j=-1)) / dy
    szz = 2.0 * mu * (W - at(W, g, 'u', k=-1)) / dz
    # shear stresses at the +1/2 edges of cell (i, j, k)
    sxy = mu_edge(i=1, j=1) * ((at(U, g, 'u', j=1) - U) / dy + (at(V, g, 'v', i=1) - V) / dx)
    sxz = mu_edge(i=1, k=1) * ((at(U, g, 'u', k=1) - U) / dz + (at(W, g, 'u', i=1) - W) / dx)
    syz = mu_edge(j=1, k=1) * ((at(V, g, 'v', k=1) - V) / dz + (at(W, g, 'u', j=1) - W) / dy)
    # the -1/2 edges in y are built from shifted velocities so that the wall ghost
    # rules apply (an edge array is never shifted across a wall)
    sxy_lo_y = mu_edge(i=1, j=-1) * ((U - at(U, g, 'u', j=-1)) / dy
                                      + (at(V, g, 'v', i=1, j=-1) - at(V, g, 'v', j=-1)) / dx)
    syz_lo_y = mu_edge(j=-1, k=1) * ((at(V, g, 'v', j=-1, k=1) - at(V, g, 'v', j=-1)) / dz
                                      + (W - at(W, g, 'u', j=-1)) / dy)
    Vx = ((at(sxx, g, 'c', i=1) - sxx) / dx + (sxy - sxy_lo_y) / dy
          + (sxz - at(sxz, g, 'c', k=-1)) / dz)
    Vy = ((sxy - at(sxy, g, 'c', i=-1)) / dx + (at(syy, g, 'c', j=1) - syy) / dy
          + (syz - at(syz, g, 'c', k=-1)) / dz)
    Vz = ((sxz - at(sxz, g, 'c', i=-1)) / dx + (syz - syz_lo_y) / dy
          + (at(szz, g, 'c', k=1) - szz) / dz)
    return Vx, Vy, Vz


def _avg4(t, g, **offs):
    """Average of a centre field over the four centres (0 or a) x (0 or b) for the
    two offsets given, e.g. ``i=1, j=-1`` -> centres (i, j), (i+1, j), (i, j-1),
    (i+1, j-1); zero-gradient ghosts at walls."""
    (k1, v1), (k2, v2) = offs.items()
    out = 0.0
    for s1 in (0, v1):
        for s2 in (0, v2):
            out = out + at(t, g, 'c', **{k1: s1, k2: s2})
    return 0.25 * out


def div_tau(tau, g):
    """div(tau) at the u, v, w faces from the six centre components (Reading 5)."""
    dx, dy, dz = g.dx, g.dy, g.dz
    txx, txy, txz, tyy, tyz, tzz = (tau[comp_index(a, b)] for a, b in
                                    ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)))
    # x-face (i+1/2, j, k): edges (i+1/2, j+-1/2), (i+1/2, k+-1/2)
    fx = ((at(txx, g, 'c', i=1) - txx) / dx
          + (_avg4(txy, g, i=1, j=1) - _avg4(txy, g, i=1, j=-1)) / dy
          + (_avg4(txz, g, i=1, k=1) - _avg4(txz, g, i=1, k=-1)) / dz)
    # y-face (i, j+1/2, k): edges (i+-1/2, j+1/2), (j+1/2, k+-1/2)
    fy = ((_avg4(txy, g, j=1, i=1) - _avg4(txy, g, j=1, i=-1)) / dx
          + (at(tyy, g, 'c', j=1) - tyy) / dy
          + (_avg4(tyz, g, j=1, k=1) - _avg4(tyz, g, j=1, k=-1)) / dz)
    # z-face (i, j, k+1/2): edges (i+-1/2, k+1/2), (j+-1/2, k+1/2)
    fz = ((_avg4(txz, g, k=1, i=1) - _avg4(txz, g, k=1, i=-1)) / dx
          + (_avg4(tyz, g, k=1, j=1) - _avg4(tyz, g, k=1, j=-1)) / dy
          + (at(tzz, g, 'c', k=1) - tzz) / dz)
    return fx, fy, fz


def grad_p(p, g):
    """grad p at the u, v, w faces (zero-gradient ghosts at walls)."""
    return ((at(p, g, 'c', i=1) - p) / g.dx,
            (at(p, g, 'c', j=1) - p) / g.dy,
            (at(p, g, 'c', k=1) - p) / g.dz)


def momentum_rhs_n(U, V, W, g, mu_s, force=None):
    """N = -div(uu) + div[mu_s(grad u + grad u^T)] + f at one time level.

    ``force`` is None or a triple of face arrays (or scalars) for the body force f."""
    Ax, Ay, Az = advection(U, V, W, g)
    Vx, Vy, Vz = viscous(U, V, W, g, mu_s)
    Nx, Ny, Nz = -Ax + Vx, -Ay + Vy, -Az + Vz
    if force is not None:
        Nx, Ny, Nz = Nx + force[0], Ny + force[1], Nz + force[2]
    return Nx, Ny, Nz
