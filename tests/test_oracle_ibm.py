"""Pins for the discrete-forcing IBM of the oracle (Eqs. IBM a-d, CoVe2): the
Roma kernel's moment conditions, exact interpolation of linear fields, momentum
conservation of the spreading, and convergence of the multi-direct iterations."""

import numpy as np

import oracle
from oracle import ibm


def test_roma_kernel_partition_of_unity_and_first_moment():
    """sum_i phi(r - i) = 1 and sum_i (r - i) phi(r - i) = 0 for any shift r, and
    sum_i phi(r - i)^2 = 1/2 (the kernel's defining conditions)."""
    for r in np.linspace(-0.5, 0.5, 41):
        i = np.arange(-3, 4)
        w = ibm.roma_phi(r - i)
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs(((r - i) * w).sum()) < 1e-14
        assert abs((w ** 2).sum() - 0.5) < 1e-14


def test_lagrangian_points_are_on_the_retracted_sphere():
    dx = 0.1
    pts, off, dvl = ibm.lagrangian_points((1.0, 0.5, 2.0), 0.8, dx)
    rr = 0.8 - 0.3 * dx
    assert np.allclose(np.linalg.norm(off, axis=1), rr, atol=1e-14)
    n = len(pts)
    assert n == round(np.pi / 3 * (12 * (rr / dx) ** 2 + 1))
    # the shell volume is shared exactly: n dV_l = 4 pi rr^2 dx + pi dx^3 / 3
    assert abs(n * dvl - (4 * np.pi * rr ** 2 * dx + np.pi * dx ** 3 / 3)) < 1e-12
    assert np.abs(off.mean(axis=0)).max() < 2.0 / n * rr    # nearly balanced


def test_interpolation_is_exact_for_linear_fields():
    """The first-moment condition makes the interpolation of a linear field exact
    on each staggered lattice (away from the periodic seam)."""
    g = oracle.Grid(16, 12, 10, 1.6, 1.2, 1.0)
    rng = np.random.default_rng(1)
    pts = rng.uniform([0.4, 0.3, 0.3], [1.2, 0.9, 0.7], size=(20, 3))
    for comp in range(3):
        xs, ys, zs, y0 = ibm._lattice(g, comp)
        F = 0.3 + 1.1 * xs[None, None, :] - 0.7 * ys[None, :, None] + 2.3 * zs[:, None, None]
        got = ibm.interpolate(F, g, comp, pts)
        want = 0.3 + 1.1 * pts[:, 0] - 0.7 * pts[:, 1] + 2.3 * pts[:, 2]
        assert np.abs(got - want).max() < 1e-12


def test_spreading_conserves_force_and_torque():
    """sum over nodes of f dV equals sum_l F_l dV_l (partition of unity), and so
    does the first moment: sum x f dV = sum X_l F_l dV_l."""
    g = oracle.Grid(20, 20, 20, 2.0, 2.0, 2.0)
    pts, off, dvl = ibm.lagrangian_points((1.0, 1.0, 1.0), 0.5, g.dx)
    rng = np.random.default_rng(2)
    Fl = rng.standard_normal(len(pts))
    cell = g.dx * g.dy * g.dz
    for comp in range(3):
        f = ibm.spread(Fl, g, comp, pts, dvl)
        assert abs(f.sum() * cell - (Fl * dvl).sum()) < 1e-12
        xs, ys, zs, y0 = ibm._lattice(g, comp)
        X = xs[None, None, :] + 0 * f
        assert abs((X * f).sum() * cell - (pts[:, 0] * Fl * dvl).sum()) < 1e-12


def test_multi_direct_forcing_drives_the_surface_velocity_to_the_target():
    """For a sphere held fixed in a uniform stream the interpolated velocity at the
    Lagrangian points approaches zero with the iterations, monotonically; the
    force opposes the stream (drag along -x on the fluid, +x on the particle)."""
    g = oracle.Grid(24, 24, 24, 2.4, 2.4, 2.4)
    star = [np.ones(g.shape), np.zeros(g.shape), np.zeros(g.shape)]
    p = {'centre': (1.2, 1.2, 1.2), 'radius': 0.4, 'u': (0, 0, 0), 'omega': (0, 0, 0)}
    pts, off, dvl = ibm.lagrangian_points(p['centre'], p['radius'], g.dx)
    errs = []
    for iters in (1, 2, 3, 6):
        us, ft = ibm.force(star, g, [p], 0.01, iters)
        errs.append(np.abs(ibm.interpolate(us[0], g, 0, pts)).max())
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 0.25 * errs[0], errs
    assert ft[0][0][0] > 0 and abs(ft[0][0][1]) < 1e-6 * ft[0][0][0]
    # a rotating sphere in fluid at rest: torque along the spin axis opposes the rotation
    q = {'centre': (1.2, 1.2, 1.2), 'radius': 0.4, 'u': (0, 0, 0), 'omega': (0, 0, 2.0)}
    us, ft = ibm.force([np.zeros(g.shape)] * 3, g, [q], 0.01, 3)
    assert ft[0][1][2] < 0 and np.abs(ft[0][0]).max() < 1e-3 * abs(ft[0][1][2])
