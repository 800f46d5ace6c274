"""Pins for the soft-particle (one-continuum, neo-Hookean) option of the oracle's
RK3 step (Sec. 3.3.2, Reading 21)."""

import numpy as np

import oracle
from paper_1803_09563_gb300 import inputs


def _case(n=16, seed=4):
    g = oracle.Grid(n, n, n, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    geo = inputs.geometry(n, n, n, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, seed, 3), 1.0)
    B = inputs.random_conformation(geo, seed + 1, amp=0.2)
    return g, U, V, W, B


def test_all_solid_equals_the_neo_hookean_step():
    """phi_s = 1 everywhere: tau = G (B - I) differs from the plain neo-Hookean
    G B by the uniform G I, whose divergence is zero; the steps agree to rounding."""
    g, U, V, W, B = _case()
    prm = oracle.Params.from_groups('neo_hookean', 1.0, 1.0, 0.5)
    a = oracle.State.rest(g, U, V, W)
    a.B = [b.copy() for b in B]
    b = a.copy()
    b.phis = np.ones(g.shape)
    b.phis_hist = np.zeros(g.shape)
    for _ in range(2):
        a = oracle.rk3_step(a, 1e-3, g, prm)
        b = oracle.rk3_step(b, 1e-3, g, prm)
    for x, y in zip([a.U, a.V, a.W] + a.B, [b.U, b.V, b.W] + b.B):
        assert np.abs(x - y).max() < 1e-13 * max(1.0, np.abs(x).max())
    assert np.abs(b.phis - 1.0).max() < 1e-14


def test_all_fluid_equals_the_newtonian_step():
    """phi_s = 0 everywhere: the stress vanishes, and u, p follow the Newtonian step
    bit for bit."""
    g, U, V, W, B = _case()
    soft = oracle.State.rest(g, U, V, W)
    soft.B = [b.copy() for b in B]
    soft.phis = np.zeros(g.shape)
    soft.phis_hist = np.zeros(g.shape)
    newt = oracle.State.rest(g, U, V, W)
    ps = oracle.Params.from_groups('neo_hookean', 1.0, 1.0, 0.5)
    pn = oracle.Params('newtonian', mu_s=ps.mu_s, mu_p=0.0, lam=1.0)
    for _ in range(2):
        soft = oracle.rk3_step(soft, 1e-3, g, ps)
        newt = oracle.rk3_step(newt, 1e-3, g, pn)
    for x, y in zip([soft.U, soft.V, soft.W, soft.p], [newt.U, newt.V, newt.W, newt.p]):
        np.testing.assert_array_equal(x, y)


def test_solid_fraction_is_carried_by_a_uniform_flow():
    """u = (1, 0, 0) in a periodic box: after one period phi_s returns to its
    initial profile to the WENO5 accuracy (the error falls ~30x per refinement)."""
    errs = []
    for n in (16, 32):
        g = oracle.Grid(n, 4, 4, 1.0, 1.0, 1.0)
        x = (np.arange(n) + 0.5) / n
        phi0 = (0.5 + 0.5 * np.sin(2 * np.pi * x))[None, None, :] + 0 * g.zeros()
        s = oracle.State.rest(g, np.ones(g.shape))
        s.phis, s.phis_hist = phi0.copy(), np.zeros(g.shape)
        prm = oracle.Params.from_groups('neo_hookean', 1.0, 1.0, 0.5)
        dt = 0.25 / n
        for _ in range(int(round(1.0 / dt))):
            s = oracle.rk3_step(s, dt, g, prm)
        errs.append(np.abs(s.phis - phi0).max())
    assert errs[1] < 3e-4 and errs[0] / errs[1] > 20, errs
