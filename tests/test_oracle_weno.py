"""Pins for the oracle's WENO5 advection derivative (Sec. 3.1)."""

import numpy as np
import pytest

import oracle
from oracle.weno import hj_weno5, weno5_one_sided


def grid1d(n, L=2 * np.pi):
    return oracle.Grid(n, 1, 1, L, 1.0, 1.0)


def test_ideal_weights_equal_textbook_fifth_order_upwind():
    """With the nonlinear weights forced to the linear ones (eps -> inf) the scheme
    must reduce to the classical 6-point fifth-order upwind-biased difference
    (-2, 15, -60, 20, 30, -3)/60 on phi_{i-3..i+2}."""
    rng = np.random.default_rng(0)
    n = 40
    phi = rng.standard_normal((1, 1, n))
    g = grid1d(n, L=float(n))          # h = 1
    dm, dp = weno5_one_sided(phi, g, 'x', eps=1e30)
    p = lambda d: np.roll(phi, -d, axis=2)
    ref_m = (-2 * p(-3) + 15 * p(-2) - 60 * p(-1) + 20 * p(0) + 30 * p(1) - 3 * p(2)) / 60.0
    ref_p = (2 * p(3) - 15 * p(2) + 60 * p(1) - 20 * p(0) - 30 * p(-1) + 3 * p(-2)) / 60.0
    np.testing.assert_allclose(dm, ref_m, rtol=0, atol=1e-12)
    np.testing.assert_allclose(dp, ref_p, rtol=0, atol=1e-12)


@pytest.mark.parametrize("c2,c1", [(0.3, -1.7), (-2.0, 0.5)])
def test_quadratic_is_exact(c2, c1):
    """On quadratic data all three smoothness indicators are equal, so the weights
    are the linear ones and the derivative is exact (default eps)."""
    v = np.arange(12, dtype=float)
    # undivided differences of phi = c2 x^2 + c1 x on unit spacing
    phi = c2 * v ** 2 + c1 * v
    d = np.diff(phi)
    i = 6
    exact = 2 * c2 * i + c1
    got = hj_weno5(d[i - 3], d[i - 2], d[i - 1], d[i], d[i + 1])
    assert abs(got - exact) < 1e-12


def test_eno_switch_at_a_jump():
    """Next to a jump the stencils that cross it get (almost) zero weight: the
    left-biased derivative one cell before a unit step, whose smooth candidate
    uses only the flat side, stays tiny instead of O(1/h)."""
    n = 32
    phi = np.zeros((1, 1, n))
    phi[..., 16:] = 1.0
    g = grid1d(n, L=float(n))
    dm, dp = weno5_one_sided(phi, g, 'x')
    # cell 14: left stencil spans 11..16, only the last difference crosses the jump
    assert abs(dm[0, 0, 14]) < 1e-6
    # cell 17: right stencil spans 15..20, only its far-downwind difference crosses
    assert abs(dp[0, 0, 17]) < 1e-6
    # and the derivative across the jump itself is O(1)
    assert dm[0, 0, 16] > 0.3


def test_convergence_order_on_smooth_data():
    """Observed order >= 4.8 for the derivative of sin(x) refined 32 -> 64 -> 128."""
    errs = []
    for n in (32, 64, 128):
        g = grid1d(n)
        x = (np.arange(n) + 0.5) * g.dx
        phi = np.sin(x)[None, None, :] + 0.0
        vel = np.ones_like(phi)
        d = oracle.weno5_derivative(phi, g, 'x', vel)
        errs.append(np.abs(d[0, 0] - np.cos(x)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() >= 4.8, (errs, orders)


def test_upwind_side_follows_velocity_sign():
    """vel > 0 takes the left-biased derivative, vel < 0 the right-biased one."""
    n = 16
    g = grid1d(n)
    phi = np.random.default_rng(1).standard_normal((1, 1, n))
    dm, dp = weno5_one_sided(phi, g, 'x')
    vel = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)[None, None, :]
    d = oracle.weno5_derivative(phi, g, 'x', vel)
    np.testing.assert_array_equal(d[..., ::2], dm[..., ::2])
    np.testing.assert_array_equal(d[..., 1::2], dp[..., 1::2])
