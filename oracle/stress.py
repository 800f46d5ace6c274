"""Stress right-hand side RT of Eqs. rt / RK-rt (Sec. 3.2.2 and 3.3.1).  TEST INFRASTRUCTURE ONLY.

RT = (a I - F B)/lambda - (u.grad B - B.grad u - grad u^T.B)

evaluated at cell centres from the face velocities and the centred B.

Reading 5 (the paper only says "second-order central differences", Sec. 3):
the centre velocity is the average of the two faces of the cell; the diagonal
gradients du/dx, dv/dy, dw/dz are the face difference across the cell; the
off-diagonal gradients are central differences of the centre velocities of the
two neighbouring cells.  u.grad B uses the WENO5 derivative upwinded by the
centre velocity (see ``weno``).
"""

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


def stress_rhs(U, V, W, B, g, prm):
    """RT of Eq. rt (AB2) / the bracket of Eq. RK-rt (RK3) at one time level."""
    uc, vc, wc = centre_velocity(U, V, W, g)
    L = velocity_gradient(U, V, W, g)
    src = rt_local(B, L, prm)
    adv = advection_B(B, uc, vc, wc, g)
    return [src[c] - adv[c] for c in range(6)]
