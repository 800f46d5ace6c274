"""Stress right-hand side RT of Eqs. rt / RK-rt (Sec. 3.2.2 and 3.3.1).  TEST INFRASTRUCTURE ONLY.

RT = (a I - F B)/lambda - (u.grad B - B.grad u - grad u^T.B)

evaluated at cell centres from the face velocities and the centred B.

Reading 5 (the paper only says "second-order central differences", Sec. 3):
the centre velocity is the average of the two faces of the cell; the diagonal
gradients du/dx, dv/dy, dw/dz are the face difference across the cell; the
off-diagonal gradients are central differences of the centre velocities of the
two neighbouring cells.  u.grad B uses the WENO5 derivative upwinded by the
centre velocity (see ``weno``).

Local artificial diffusion (Sec. 3.1, Reading 16): where B has lost positive
definiteness (det B < 0) or, for FENE-P, where tr B has reached 95 % of L^2,
art_diff times the 7-point Laplacian of B (zero-gradient ghosts at walls) is
added to RT.  The cells are selected from the B the right-hand side is formed
from, so the term takes the time-integration weights of RT.
"""

import numpy as np


from .grid import at
from .models import rt_local
from .weno import weno5_derivative


def centre_velocity(U, V, W, g):
    """Cell-centre velocity: mean of the two faces of each cell."""
    uc = 0.5 * (U + at(U, g, 'u', i=-1))
    vc = 0.5 * (V + at(V, g, 'v', j=-1))
    wc = 0.5 * (W + at(W, g, 'u', k=-1))
    return uc, vc, wc


def velocity_gradient(U, V, W, g):
    """L[i][j] = du_i/dx_j at cell centres (Reading 5)."""
    uc, vc, wc = centre_velocity(U, V, W, g)
    dx, dy, dz = g.dx, g.dy, g.dz

    def cdx(f, kind):
        return (at(f, g, kind, i=1) - at(f, g, kind, i=-1)) / (2.0 * dx)

    def cdy(f, kind):
        return (at(f, g, kind, j=1) - at(f, g, kind, j=-1)) / (2.0 * dy)

    def cdz(f, kind):
        return (at(f, g, kind, k=1) - at(f, g, kind, k=-1)) / (2.0 * dz)

    Lxx = (U - at(U, g, 'u', i=-1)) / dx
    Lyy = (V - at(V, g, 'v', j=-1)) / dy
    Lzz = (W - at(W, g, 'u', k=-1)) / dz
    # uc and wc are centred in y like u and w: odd (no-slip) ghosts at walls
    Lxy = cdy(uc, 'u')
    Lxz = cdz(uc, 'u')
    Lyx = cdx(vc, 'c')
    Lyz = cdz(vc, 'c')
    Lzx = cdx(wc, 'u')
    Lzy = cdy(wc, 'u')
    return [[Lxx, Lxy, Lxz], [Lyx, Lyy, Lyz], [Lzx, Lzy, Lzz]]


def advection_B(B, uc, vc, wc, g):
    """u.grad B for the six components, WENO5 upwinded per direction."""
    out = []
    for c in range(6):
        out.append(uc * weno5_derivative(B[c], g, 'x', uc)
                   + vc * weno5_derivative(B[c], g, 'y', vc)
                   + wc * weno5_derivative(B[c], g, 'z', wc))
    return out


def determinant(B):
    """det of the symmetric tensor stored as (xx, xy, xz, yy, yz, zz), by cofactors
    along the first row."""
    xx, xy, xz, yy, yz, zz = B
    return xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz)


def diffusion_cells(B, prm):
    """Boolean mask of the cells that receive the artificial diffusion (Sec. 3.1)."""
    mask = determinant(B) < 0.0
    if prm.model == 'fene_p':
        mask = mask | (B[0] + B[3] + B[5] >= 0.95 * prm.L2)
    return mask


def centre_laplacian(f, g):
    """7-point Laplacian of a centred field with the copy ghost rule."""
    return ((at(f, g, 'c', i=1) - 2.0 * f + at(f, g, 'c', i=-1)) / g.dx ** 2
            + (at(f, g, 'c', j=1) - 2.0 * f + at(f, g, 'c', j=-1)) / g.dy ** 2
            + (at(f, g, 'c', k=1) - 2.0 * f + at(f, g, 'c', k=-1)) / g.dz ** 2)


def stress_rhs(U, V, W, B, g, prm):
    """RT of Eq. rt (AB2) / the bracket of Eq. RK-rt (RK3) at one time level."""
    uc, vc, wc = centre_velocity(U, V, W, g)
    L = velocity_gradient(U, V, W, g)
    src = rt_local(B, L, prm)
    adv = advection_B(B, uc, vc, wc, g)
    rt = [src[c] - adv[c] for c in range(6)]
    if getattr(prm, 'art_diff', 0.0) > 0.0:
        mask = diffusion_cells(B, prm)
        rt = [rt[c] + np.where(mask, prm.art_diff * centre_laplacian(B[c], g), 0.0) for c in range(6)]
    return rt
