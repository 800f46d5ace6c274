"""Pins for the implicit (Crank-Nicolson within the RK3 substep) viscous option of
the oracle (Eq. NS-num1 read literally): the Helmholtz solve against the
oracle's own Laplacian, and the closed-form decay of shear modes."""

import numpy as np
import pytest

import oracle
from oracle.momentum import laplacian
from oracle.poisson import solve_helmholtz


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("kind", ['u', 'v'])
def test_helmholtz_solution_satisfies_the_operator(walls, kind):
    """x - c lap(x) = r with lap the 7-point Laplacian and the component's ghost
    rule (brute-force residual); with walls the v unknowns are rows 0..ny-2 and
    the top face stays zero."""
    g = oracle.Grid(12, 10, 8, 1.3, 2.0, 0.9, walls)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(g.shape)
    if walls and kind == 'v':
        r[:, -1, :] = 0.0
    c = 0.037
    x = solve_helmholtz(r, g, c, kind)
    res = x - c * laplacian(x, g, kind) - r
    rows = slice(0, g.ny - 1) if (walls and kind == 'v') else slice(None)
    assert np.abs(res[:, rows, :]).max() < 1e-12 * np.abs(r).max()
    if walls and kind == 'v':
        assert np.abs(x[:, -1, :]).max() == 0.0


def _decay(lam, nu, dt):
    f = 1.0
    for a in oracle.RK3_ALPHA:
        f *= (1.0 - a * dt * nu * lam) / (1.0 + a * dt * nu * lam)
    return f


def test_periodic_shear_mode_decays_by_the_crank_nicolson_factor():
    """u = sin(2 pi m z / lz): no advection, no pressure; one implicit-viscous RK3
    step multiplies it by prod_k (1 - a_k dt nu lam)/(1 + a_k dt nu lam),
    lam = (2 - 2 cos(2 pi m/nz))/dz^2."""
    g = oracle.Grid(8, 8, 24, 1.0, 1.0, 2.0)
    m, nu, dt = 3, 0.2, 0.05
    U = np.sin(2 * np.pi * m * (np.arange(g.nz) + 0.5) / g.nz)[:, None, None] + 0 * g.zeros()
    s = oracle.State.rest(g, U)
    prm = oracle.Params('newtonian', mu_s=nu, mu_p=0.0, lam=1.0)
    out = oracle.rk3_step(s, dt, g, prm, implicit_viscous=True)
    lam = (2 - 2 * np.cos(2 * np.pi * m / g.nz)) / g.dz ** 2
    np.testing.assert_allclose(out.U, U * _decay(lam, nu, dt), rtol=0, atol=1e-13)
    assert np.abs(out.V).max() < 1e-14 and np.abs(out.W).max() < 1e-14


def test_channel_shear_mode_decays_by_the_crank_nicolson_factor():
    """Between no-slip walls u_j = sin(pi m (j + 1/2)/ny) is an eigenvector of the
    discrete Laplacian with the odd-mirror ghosts, eigenvalue
    -(2 - 2 cos(pi m/ny))/dy^2 (checked), and decays by the same factor."""
    g = oracle.Grid(8, 20, 8, 1.0, 2.0, 1.0, True)
    m, nu, dt = 2, 0.1, 0.02
    U = np.sin(np.pi * m * (np.arange(g.ny) + 0.5) / g.ny)[None, :, None] + 0 * g.zeros()
    lam = (2 - 2 * np.cos(np.pi * m / g.ny)) / g.dy ** 2
    np.testing.assert_allclose(laplacian(U, g, 'u'), -lam * U, rtol=0, atol=1e-10)
    s = oracle.State.rest(g, U)
    prm = oracle.Params('newtonian', mu_s=nu, mu_p=0.0, lam=1.0)
    out = oracle.rk3_step(s, dt, g, prm, implicit_viscous=True)
    np.testing.assert_allclose(out.U, U * _decay(lam, nu, dt), rtol=0, atol=1e-13)


def test_implicit_and_explicit_viscous_steps_agree_to_second_order():
    """Both steps are consistent to second order, so on a smooth Taylor-Green box
    one step of each differs by the local error O(dt^3): halving dt cuts the
    difference about eight times."""
    n = 16
    g = oracle.Grid(n, n, n, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    U = np.sin(g.xf()) * np.cos(g.yc()) * np.cos(g.zc())
    V = -np.cos(g.xc()) * np.sin(g.yf()) * np.cos(g.zc())
    prm = oracle.Params.from_groups('oldroyd_b', 1.0, 1.0, 0.5)
    diffs = []
    for dt in (0.02, 0.01):
        a = oracle.rk3_step(oracle.State.rest(g, U, V, g.zeros()), dt, g, prm)
        b = oracle.rk3_step(oracle.State.rest(g, U, V, g.zeros()), dt, g, prm, implicit_viscous=True)
        diffs.append(np.abs(a.U - b.U).max())
    assert 6.5 < diffs[0] / diffs[1] < 10.5, diffs
