"""Pins for the local artificial diffusion of the conformation tensor (Sec. 3.1):
the cells it acts on (det B < 0; tr B >= 0.95 L^2 for FENE-P) and the size of the
term (art_diff times the 7-point Laplacian), checked against closed forms."""

import numpy as np

import oracle


def _fields(g, B):
    zero = g.zeros()
    return zero, zero.copy(), zero.copy(), B


def _rhs(g, B, model='oldroyd_b', art=0.0, L2=0.0):
    prm = oracle.Params.from_groups(model, 1.0, 1.0, 0.5, L2=L2, art_diff=art)
    U, V, W, B = _fields(g, B)
    return oracle.stress_rhs(U, V, W, B, g, prm)


def _eig(m, n, h):
    """Eigenvalue of the 1-D second difference for the mode sin(2 pi m i / n):
    (2 - 2 cos(2 pi m / n)) / h^2."""
    return (2.0 - 2.0 * np.cos(2.0 * np.pi * m / n)) / h ** 2


def test_off_and_unflagged_cells_leave_rt_unchanged():
    """art_diff = 0, or an SPD tensor below the trace limit, changes nothing (bitwise)."""
    g = oracle.Grid(12, 10, 8, 1.0, 1.0, 1.0)
    rng = np.random.default_rng(3)
    S = [0.2 * rng.standard_normal(g.shape) for _ in range(6)]
    B = [S[c] + (1.5 if c in (0, 3, 5) else 0.0) for c in range(6)]
    assert oracle.determinant(B).min() > 0
    base = _rhs(g, B, 'fene_p', 0.0, L2=60.0)
    for x, y in zip(base, _rhs(g, B, 'fene_p', 0.7, L2=60.0)):
        np.testing.assert_array_equal(x, y)


def test_sine_modes_take_the_discrete_laplacian_eigenvalues():
    """With det B < 0 everywhere every cell is diffused.  B_xx = -1 plus three sine
    modes (one per direction) gains exactly -kappa * (a lx + b ly + c lz) per mode,
    l = (2 - 2 cos(2 pi m/n))/h^2; the constant components gain nothing."""
    nx, ny, nz = 16, 12, 18
    g = oracle.Grid(nx, ny, nz, 2.0, 1.5, 3.0)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    sx, sy, sz = np.sin(2 * np.pi * 3 * i / nx), np.sin(2 * np.pi * 2 * j / ny), np.sin(2 * np.pi * 5 * k / nz)
    a, b, c = 0.1, 0.05, 0.02
    B = [g.zeros() for _ in range(6)]
    B[0] = -1.0 + a * sx + b * sy + c * sz + 0 * g.zeros()
    B[3] = B[3] + 1.0
    B[5] = B[5] + 1.0
    assert oracle.determinant(B).max() < 0
    kappa = 0.3
    d = [x - y for x, y in zip(_rhs(g, B, art=kappa), _rhs(g, B))]
    want = -kappa * (a * _eig(3, nx, g.dx) * sx + b * _eig(2, ny, g.dy) * sy + c * _eig(5, nz, g.dz) * sz)
    assert np.abs(d[0] - want).max() < 1e-12 * np.abs(want).max() * 100
    for comp in (1, 2, 3, 4, 5):
        assert np.abs(d[comp]).max() == 0.0
    # all cells diffused on a periodic grid: the term sums to zero
    assert abs(d[0].sum()) < 1e-10 * np.abs(d[0]).max()


def test_fene_p_trace_threshold_at_95_percent_of_L2():
    """tr B = 0.951 L^2 is diffused, tr B = 0.949 L^2 is not; the Oldroyd-B model has
    no trace trigger."""
    g = oracle.Grid(8, 8, 8, 1.0, 1.0, 1.0)
    L2 = 60.0
    rng = np.random.default_rng(5)
    frac = np.where(rng.random(g.shape) < 0.5, 0.951, 0.949)
    iso = frac * L2 / 3.0
    B = [iso, 0.01 * rng.standard_normal(g.shape), g.zeros(), iso.copy(), g.zeros(), iso.copy()]
    assert oracle.determinant(B).min() > 0
    d = [x - y for x, y in zip(_rhs(g, B, 'fene_p', 0.5, L2), _rhs(g, B, 'fene_p', 0.0, L2))]
    hit = frac > 0.95
    lap = oracle.stress.centre_laplacian(B[1], g)
    np.testing.assert_allclose(d[1][hit], 0.5 * lap[hit], rtol=1e-12, atol=1e-12)
    assert np.abs(d[1][~hit]).max() == 0.0 and np.abs(d[0][~hit]).max() == 0.0
    np.testing.assert_array_equal(oracle.diffusion_cells(B, oracle.Params('oldroyd_b', 0.5, 0.5, 1.0, L2=L2)),
                                  np.zeros(g.shape, bool))


def test_wall_rows_use_the_zero_gradient_ghost():
    """Walls at y = +-ly/2: for B_xx = -1 + f(y) the first and last rows see the
    one-sided second difference (f_1 - f_0)/dy^2 and (f_{n-2} - f_{n-1})/dy^2."""
    g = oracle.Grid(8, 10, 8, 1.0, 2.0, 1.0, True)
    f = np.linspace(0.0, 0.3, g.ny) ** 2
    B = [g.zeros() for _ in range(6)]
    B[0] = -1.0 + f[None, :, None] + g.zeros()
    B[3] = B[3] + 1.0
    B[5] = B[5] + 1.0
    kappa = 0.2
    d = _rhs(g, B, art=kappa)[0] - _rhs(g, B)[0]
    dy2 = g.dy ** 2
    want = np.empty(g.ny)
    want[0] = (f[1] - f[0]) / dy2
    want[-1] = (f[-2] - f[-1]) / dy2
    want[1:-1] = (f[2:] - 2 * f[1:-1] + f[:-2]) / dy2
    np.testing.assert_allclose(d[0, :, 0], kappa * want, rtol=1e-12, atol=1e-13)
