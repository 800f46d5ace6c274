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


def ab2_predictor(g, tp, dt, U, V, W, p, B, phi_next, starts, widths):
    """Oracle (u*, B^{n+1}) of the first AB2 step (steps 2-4 of ``oracle.ab2``: no
    history) on the window at ``starts``, from the full-size level set phi^{n+1}
    (the level set's own advection reaches 9 cells, and a mass shift is global, so
    phi^{n+1} is computed on the full fields and only cut here).  The mixture
    properties, the interface force and the AB2 predictor reach 3 cells of
    phi^{n+1} and the same distances as the RK3 predictor in (u, p, B); the one
    global quantity, the mean that makes the buoyancy mean-free, is taken from the
    full phi^{n+1}.  Returns
    (compared index, u* triple, B^{n+1} list, B^n list, phi^{n+1}), all on the
    window."""
    from oracle.ab2 import ab2_predictor as predict
    from oracle import levelset as ls
    # the buoyancy is made mean-free with the mean over the whole domain
    b_mean = float((1.0 - ls.heaviside(phi_next, tp.eps_cells * g.dx)).mean()) * tp.drho_g
    gw = window_grid(g, widths)
    c = lambda a: cut(a, starts, widths)
    st = oracle.State.rest(gw, c(U), c(V), c(W))
    st.p = c(p)
    st.B = [c(b) for b in B]
    phw = c(phi_next)
    star, Bn, _, _, _ = predict(st, phw, dt, gw, tp, 0, b_mean)
    return interior(widths, st.U.shape), star, Bn, st.B, phw
