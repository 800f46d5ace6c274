"""The oracle on windows cut from full-size fields (sampled parity at full size).

The stress update and the momentum predictor of one RK3 substep (Eqs. rk3tau,
NS-num1, rk3) are local.  A cell's B^k depends on B^{k-1} within 3 cells (the WENO5
stencils of Sec. 3.1) and on the velocity within 2 (centre velocity and gradient).
A face's u* depends on u within 2 (advection, viscous term) and on p, B^{k-1} and
B^k within 2 (grad p; div tau through edge averages, Reading 5), so on B^{k-1}
within 5.  A window of w cells along a periodic direction, cut with the periodic
wrap and handed to the oracle as a periodic box of w cells, therefore reproduces
the full-size values at every cell at least MARGIN cells from its cut faces.
Wall-bounded directions are kept whole, so their wall rules apply unchanged.
"""

import numpy as np

import oracle

MARGIN = 7


def _axis_index(n, start, width):
    return np.arange(n) if width is None else (start + np.arange(width)) % n


def cut(a, starts, widths):
    """Window of a [nz][ny][nx] array (or a scalar, returned as is).  ``starts`` and
    ``widths`` are (x, y, z); a width of None keeps the whole axis."""
    if np.ndim(a) == 0:
        return a
    nz, ny, nx = np.shape(a)
    iz = _axis_index(nz, starts[2], widths[2])
    iy = _axis_index(ny, starts[1], widths[1])
    ix = _axis_index(nx, starts[0], widths[0])
    return np.asarray(a)[np.ix_(iz, iy, ix)]


def window_grid(g, widths):
    """The oracle grid of a window: the same spacings, w cells per cut axis."""
    wx = g.nx if widths[0] is None else widths[0]
    wy = g.ny if widths[1] is None else widths[1]
    wz = g.nz if widths[2] is None else widths[2]
    return oracle.Grid(wx, wy, wz, wx * g.dx, wy * g.dy, wz * g.dz, g.walls)


def interior(widths, shape):
    """Index of the window cells at least MARGIN from every cut face ([z][y][x])."""
    out = []
    for w, n in ((widths[2], shape[0]), (widths[1], shape[1]), (widths[0], shape[2])):
        out.append(slice(None) if w is None else slice(MARGIN, w - MARGIN))
    return tuple(out)


def predictor(g, prm, dt, k, U, V, W, p, B, starts, widths, force=None):
    """Oracle (u*, B^k) of RK3 substep k (the first substep has no history terms) on
    the window at ``starts``; returns (compared index, u* triple, B^k list, B^{k-1}
    list), all on the window."""
    assert k == 0, "windows carry no RK3 history"
    gw = window_grid(g, widths)
    c = lambda a: cut(a, starts, widths)
    st = oracle.State.rest(gw, c(U), c(V), c(W))
    st.p = c(p)
    st.B = [c(b) for b in B]
    fw = None if force is None else tuple(c(f) for f in force)
    star, Bn = oracle.rk3_substep(st, k, dt, gw, prm, fw, predictor_only=True)
    return interior(widths, st.U.shape), star, Bn, st.B
