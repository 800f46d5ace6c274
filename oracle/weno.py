"""Fifth-order WENO for the advection term u.grad(B) (Sec. 3.1).  TEST INFRASTRUCTURE ONLY.

The paper replaces the compact upwind scheme by an explicit fifth-order WENO
scheme (Liu-Osher-Chan) for the advection terms of Eqs. SRM2, ls-adv and reinit.
Reading 4: the advection is non-conservative (u.grad B with u at the cell
centre), so the scheme is taken in Hamilton-Jacobi form -- the derivative at a
cell centre is a convex combination of the three third-order candidate
derivatives built from undivided first differences, weighted with the Jiang-Shu
smoothness indicators, linear weights (1/10, 6/10, 3/10), eps = 1e-6 on the
undivided differences and power 2.  The upwind side is chosen by the sign of
the centre velocity; a zero velocity contributes nothing.
"""

import numpy as np

from .grid import at

WENO_EPS = 1.0e-6


def hj_weno5(v1, v2, v3, v4, v5, eps=WENO_EPS):
    """WENO5 combination of five consecutive undivided differences.

    v1..v5 are ordered from the far upwind side towards the downwind side; the
    result is the undivided derivative (divide by h for d/dx).
    """
    # three third-order candidates (Sec. 3.1, WENO of Liu-Osher-Chan)
    q1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0
    q2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0
    q3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0
    # smoothness indicators
    s1 = 13.0 / 12.0 * (v1 - 2.0 * v2 + v3) ** 2 + 0.25 * (v1 - 4.0 * v2 + 3.0 * v3) ** 2
    s2 = 13.0 / 12.0 * (v2 - 2.0 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
    s3 = 13.0 / 12.0 * (v3 - 2.0 * v4 + v5) ** 2 + 0.25 * (3.0 * v3 - 4.0 * v4 + v5) ** 2
    # nonlinear weights from the linear weights (1/10, 6/10, 3/10)
    a1 = 0.1 / (eps + s1) ** 2
    a2 = 0.6 / (eps + s2) ** 2
    a3 = 0.3 / (eps + s3) ** 2
    asum = a1 + a2 + a3
    return (a1 * q1 + a2 * q2 + a3 * q3) / asum


def weno5_one_sided(phi, g, axis, eps=WENO_EPS):
    """Left-biased (upwind for a positive velocity) and right-biased derivatives of a
    cell-centred field along ``axis`` ('x', 'y' or 'z'), zero-gradient ghosts at walls."""
    h = {'x': g.dx, 'y': g.dy, 'z': g.dz}[axis]

    def p(d):
        return at(phi, g, 'c', **{{'x': 'i', 'y': 'j', 'z': 'k'}[axis]: d})

    pm3, pm2, pm1, p0, pp1, pp2, pp3 = (p(d) for d in (-3, -2, -1, 0, 1, 2, 3))
    dm = hj_weno5(pm2 - pm3, pm1 - pm2, p0 - pm1, pp1 - p0, pp2 - pp1, eps) / h
    dp = hj_weno5(pp3 - pp2, pp2 - pp1, pp1 - p0, p0 - pm1, pm1 - pm2, eps) / h
    return dm, dp


def weno5_derivative(phi, g, axis, vel, eps=WENO_EPS):
    """Upwind WENO5 derivative of ``phi`` along ``axis`` for the centre velocity ``vel``."""
    dm, dp = weno5_one_sided(phi, g, axis, eps)
    return np.where(vel > 0.0, dm, dp)
