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


def test_inner_integrals_of_uniform_and_rigid_fields():
    """For u = const the integrals are the sampled particle volume times u (and
    about zero moment); for a rigid rotation u = omega x r about the centre the
    angular integral is the sampled moment of inertia, close to 2/5 V R^2 omega."""
    g = oracle.Grid(32, 32, 32, 2.0, 2.0, 2.0)
    c, R = (1.0, 1.03, 0.97), 0.45
    ones, zero = np.ones(g.shape), np.zeros(g.shape)
    Iu, Ir = ibm.inner_integrals(0.7 * ones, zero, -0.2 * ones, g, c, R)
    vol = 4 / 3 * np.pi * R ** 3
    assert abs(Iu[0] / 0.7 - vol) < 0.01 * vol and abs(Iu[2] / -0.2 - vol) < 0.01 * vol and Iu[1] == 0.0
    assert np.abs(Ir).max() < 1e-3 * vol
    # rigid rotation about z through the centre, sampled on each lattice
    om = 1.3
    xs, ys, zs, y0 = ibm._lattice(g, 0)
    Uz = -om * (ys[None, :, None] - c[1]) + 0 * g.zeros()
    xs, ys, zs, y0 = ibm._lattice(g, 1)
    Vz = om * (xs[None, None, :] - c[0]) + 0 * g.zeros()
    Iu, Ir = ibm.inner_integrals(Uz, Vz, zero, g, c, R)
    assert abs(Ir[2] - 0.4 * vol * R * R * om) < 0.03 * 0.4 * vol * R * R * om
    assert np.abs(Iu).max() < 1e-3 * vol


def test_free_particle_first_substep_under_gravity():
    """A heavy sphere at rest in fluid at rest: in the first substep the IBM force
    and the inner-fluid integrals vanish, so U^1 = dt_s (1 - 1/rho) g and
    X^1 = X^0 + dt_s U^1 / 2 (closed form)."""
    g = oracle.Grid(24, 24, 24, 2.4, 2.4, 2.4)
    p = {'centre': (1.2, 1.2, 1.2), 'radius': 0.4, 'u': (0, 0, 0), 'omega': (0, 0, 0), 'rho': 2.5}
    s = oracle.State.rest(g)
    s.particles = [p]
    prm = oracle.Params.from_groups('newtonian', 10.0, 1.0, 1.0)
    out = oracle.rk3_substep(s, 0, 0.01, g, prm, gravity=9.81)
    dts = 2 * oracle.RK3_ALPHA[0] * 0.01
    uy = -dts * (1 - 1 / 2.5) * 9.81
    q = out.particles[0]
    assert abs(q['u'][1] - uy) < 1e-14 and abs(q['u'][0]) < 1e-14 and abs(q['u'][2]) < 1e-14
    assert abs(q['centre'][1] - (1.2 + 0.5 * dts * uy)) < 1e-14


def test_neutrally_buoyant_sphere_in_uniform_flow_keeps_its_velocity():
    """rho_p = rho_f, u = U everywhere and U_p = U: the forcing and the change of
    the inner integrals vanish, so the particle keeps U and the flow is unchanged."""
    g = oracle.Grid(24, 24, 24, 2.4, 2.4, 2.4)
    U0 = (0.3, -0.1, 0.2)
    s = oracle.State.rest(g, U0[0] + 0 * g.zeros(), U0[1] + 0 * g.zeros(), U0[2] + 0 * g.zeros())
    s.particles = [{'centre': (1.2, 1.2, 1.2), 'radius': 0.4, 'u': U0, 'omega': (0, 0, 0), 'rho': 1.0}]
    prm = oracle.Params.from_groups('newtonian', 10.0, 1.0, 1.0)
    out = oracle.rk3_step(s, 0.01, g, prm)
    assert np.abs(np.asarray(out.particles[0]['u']) - U0).max() < 1e-12
    assert np.abs(np.asarray(out.particles[0]['omega'])).max() < 1e-12
    assert np.abs(out.U - U0[0]).max() < 1e-12 and np.abs(out.V - U0[1]).max() < 1e-12
