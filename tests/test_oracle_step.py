"""Pins for the oracle's whole RK3 step (Sec. 3.3.1): exact Navier-Stokes solutions,
steady channel flow of an Oldroyd-B fluid, projection bound and discrete symmetries."""

import numpy as np
import pytest

import oracle
from paper_1803_09563_gb300 import inputs


def taylor_green_2d_error(n, dt, T, nu=0.1):
    g = oracle.Grid(n, n, 4, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    U = np.sin(g.xf()) * np.cos(g.yc()) + 0 * g.zeros()
    V = -np.cos(g.xc()) * np.sin(g.yf()) + 0 * g.zeros()
    prm = oracle.Params('newtonian', mu_s=nu, mu_p=0.0, lam=1.0)
    s = oracle.State.rest(g, U, V, g.zeros())
    s.p = 0.25 * (np.cos(2 * g.xc()) + np.cos(2 * g.yc())) + 0 * g.zeros()
    for _ in range(int(round(T / dt))):
        s = oracle.rk3_step(s, dt, g, prm)
    decay = np.exp(-2 * nu * T)
    return np.abs(s.U - U * decay).max(), s, g


def test_taylor_green_decay_second_order_in_space():
    """2D Taylor-Green vortex u = sin x cos y e^{-2 nu t} is an exact Navier-Stokes
    solution; the error of the central-difference step falls ~4x per refinement."""
    e16, _, _ = taylor_green_2d_error(16, 0.02, 0.4)
    e32, s, g = taylor_green_2d_error(32, 0.01, 0.4)
    assert e32 < 3e-4 and e16 / e32 > 3.6, (e16, e32)
    assert np.abs(oracle.divergence(s.U, s.V, s.W, g)).max() < 1e-12


def test_oldroyd_b_poiseuille_steady_state():
    """Start-up Poiseuille flow of an Oldroyd-B fluid (Sec. 4.1.1) reaches the steady
    state u = (G/2 mu_0)(1 - y^2) (to the O(dy^2) of the wall treatment), with
    tau_xy = mu_p du/dy and tau_xx = 2 lambda mu_p (du/dy)^2 holding exactly for the
    discrete gradient."""
    g = oracle.Grid(1, 8, 1, 1.0, 2.0, 1.0, True)
    prm = oracle.Params.from_groups('oldroyd_b', 1.0, 0.25, 0.5)
    s = oracle.State.rest(g)
    for _ in range(500):
        s = oracle.rk3_step(s, 0.012, g, prm, (2.0, 0.0, 0.0))
    y = g.yc()[0, :, 0]
    assert np.abs(s.U[0, :, 0] - (1 - y ** 2)).max() < 0.05
    L = oracle.velocity_gradient(s.U, s.V, s.W, g)
    tau = oracle.tau_from_B(s.B, prm)
    assert np.abs(tau[1] - prm.mu_p * L[0][1]).max() < 1e-6
    assert np.abs(tau[0] - 2 * prm.lam * prm.mu_p * L[0][1] ** 2).max() < 1e-6
    assert np.abs(s.V).max() == 0.0


def c1_state():
    n = 32
    geo = inputs.geometry(n, n, n, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    g = oracle.Grid(n, n, n, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    U, V, W = inputs.taylor_green(geo)
    return g, oracle.State.rest(g, U, V, W)


def test_c1_energy_decays_divergence_free_and_mirror_symmetric():
    """Single-phase Oldroyd-B Taylor-Green box: kinetic energy decreases, the
    projected field has max|div u| <= 1e-12, and the mirror symmetry
    u(x) = -u(2 pi - x) of the initial field is kept to round-off."""
    g, s = c1_state()
    prm = oracle.Params.from_groups('oldroyd_b', 1.0, 1.0, 0.5)
    E = [0.5 * (s.U ** 2 + s.V ** 2 + s.W ** 2).mean()]
    for _ in range(2):
        s = oracle.rk3_step(s, 1e-3, g, prm)
        E.append(0.5 * (s.U ** 2 + s.V ** 2 + s.W ** 2).mean())
        assert np.abs(oracle.divergence(s.U, s.V, s.W, g)).max() <= 1e-12
    assert E[0] > E[1] > E[2]
    n = g.nx
    # face i+1/2 at (i+1)h mirrors to face n-i-2; centre i mirrors to n-1-i
    mir_face = (n - 2 - np.arange(n)) % n
    mir_cell = n - 1 - np.arange(n)
    assert np.abs(s.U + s.U[:, :, mir_face]).max() < 1e-12
    assert np.abs(s.V - s.V[:, :, mir_cell]).max() < 1e-12
    assert np.abs(s.B[1] + s.B[1][:, :, mir_cell]).max() < 1e-12
    assert np.abs(s.B[0] - s.B[0][:, :, mir_cell]).max() < 1e-12


def test_saramito_bi_zero_step_equals_oldroyd_b_step():
    g, s = c1_state()
    a = oracle.rk3_step(s.copy(), 1e-3, g, oracle.Params.from_groups('oldroyd_b', 1.0, 1.0, 0.5))
    b = oracle.rk3_step(s.copy(), 1e-3, g, oracle.Params.from_groups('saramito', 1.0, 1.0, 0.5, Bi=0.0))
    for x, y in zip([a.U, a.V, a.W, a.p] + a.B, [b.U, b.V, b.W, b.p] + b.B):
        np.testing.assert_array_equal(x, y)


def test_rest_state_with_identity_conformation_stays_at_rest():
    """u = 0, B = I is an exact steady state for every model (tau = 0)."""
    g = oracle.Grid(8, 8, 8, 1.0, 1.0, 1.0)
    for model, extra in (('oldroyd_b', {}), ('fene_p', {'L2': 100.0}), ('saramito', {'Bi': 0.3})):
        prm = oracle.Params.from_groups(model, 1.0, 1.0, 0.5, **extra)
        s = oracle.rk3_step(oracle.State.rest(g), 1e-2, g, prm)
        assert np.abs(s.U).max() == 0.0 and np.abs(s.p).max() == 0.0
        for c, b in enumerate(s.B):
            assert np.abs(b - (1.0 if c in (0, 3, 5) else 0.0)).max() < 1e-15


def test_volume_penalisation_limits():
    """Eq. forceAdded: alpha = 0 leaves the step unchanged (bitwise); alpha = 1 on
    every face gives u** = 0 before the projection, hence u = 0 after it; and a
    fixed solid block in a driven channel keeps the velocity inside it small
    compared with the bulk flow."""
    g, s = c1_state()
    prm = oracle.Params.from_groups('oldroyd_b', 1.0, 1.0, 0.5)
    zero = (g.zeros(), g.zeros(), g.zeros())
    a = oracle.rk3_step(s.copy(), 1e-3, g, prm)
    b = oracle.rk3_step(s.copy(), 1e-3, g, prm, solid=zero)
    for x, y in zip([a.U, a.V, a.W, a.p] + a.B, [b.U, b.V, b.W, b.p] + b.B):
        np.testing.assert_array_equal(x, y)
    one = tuple(np.ones(g.shape) for _ in range(3))
    c = oracle.rk3_substep(s.copy(), 0, 1e-3, g, prm, solid=one)
    assert max(np.abs(c.U).max(), np.abs(c.V).max(), np.abs(c.W).max()) == 0.0
    # channel with a solid block in its middle
    geo = inputs.geometry(16, 16, 8, 4.0, 2.0, 2.0, True)
    gc = oracle.Grid(16, 16, 8, 4.0, 2.0, 2.0, True)
    block = lambda x, y, z: ((np.abs(x - 2.0) < 0.5) & (np.abs(y) < 0.5)).astype(float)
    al = inputs.solid_fractions(geo, block)
    U, V, W = inputs.poiseuille(geo)
    st = oracle.State.rest(gc, U, V, W)
    pr = oracle.Params.from_groups('newtonian', 10.0, 1.0, 1.0)
    for _ in range(40):
        st = oracle.rk3_step(st, 5e-3, gc, pr, (0.2, 0.0, 0.0), al)
    solid = al[0] > 0.99
    assert np.abs(st.U[solid]).max() < 0.05 * np.abs(st.U).max()
    assert np.abs(oracle.divergence(st.U, st.V, st.W, gc)).max() < 1e-12


def test_solid_fractions_of_a_block():
    """The sub-sampled fractions integrate to the block's volume and are exactly
    0 / 1 away from its surface."""
    geo = inputs.geometry(16, 16, 16, 2.0, 2.0, 2.0)
    block = lambda x, y, z: ((np.abs(x - 1.0) < 0.4) & (np.abs(y - 1.0) < 0.3) & (np.abs(z - 1.0) < 0.5)).astype(float)
    for a in inputs.solid_fractions(geo, block, samples=8):
        vol = a.sum() * (2.0 / 16) ** 3
        assert abs(vol - 0.8 * 0.6 * 1.0) < 0.02
        assert set(np.unique(a[(a > 0) & (a < 1)]).round(6)) <= set((np.arange(1, 512) / 512).round(6))


@pytest.mark.parametrize("walls,m,dt", [(False, 2, 0.01), (False, 3, 0.002), (True, 1, 5e-4), (True, 3, 1e-4)])
def test_shear_mode_decays_by_the_rk3_stability_polynomial(walls, m, dt):
    """A shear mode u = f(y) e_x is an exact Navier-Stokes solution (no advection,
    no pressure) whose discrete form decays as u' = -nu lambda u, lambda the
    eigenvalue of the discrete Laplacian: (2 - 2 cos(m dy)) / dy^2 for sin(m y)
    (periodic) and (2 - 2 cos(m pi / ny)) / dy^2 for sin(m pi (j + 1/2) / ny) between
    no-slip walls.  One step of the three-substep scheme of Eq. RK (viscous term
    explicit with the weights zeta, xi, Reading 3) multiplies it by the stability
    polynomial of a three-stage third-order method, 1 + z + z^2/2 + z^3/6 with
    z = -nu lambda dt, to rounding; a wrong RK3 weight changes the polynomial."""
    nx, ny, nz = 8, 16, 6
    ly = 2.0 if walls else 2 * np.pi
    g = oracle.Grid(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
    if walls:
        prof = np.sin(m * np.pi * (np.arange(ny) + 0.5) / ny)
        lam = (2.0 - 2.0 * np.cos(m * np.pi / ny)) / g.dy ** 2
    else:
        prof = np.sin(m * g.yc()).ravel()
        lam = (2.0 - 2.0 * np.cos(m * g.dy)) / g.dy ** 2
    U = np.broadcast_to(prof[None, :, None], g.shape).copy()
    prm = oracle.Params('newtonian', mu_s=2.0, mu_p=0.0, lam=1.0)
    s1 = oracle.rk3_step(oracle.State.rest(g, U), dt, g, prm)
    z = -prm.mu_s * lam * dt
    amp = 1.0 + z + z * z / 2.0 + z ** 3 / 6.0
    assert abs(z) > 1e-4
    assert np.abs(s1.U - amp * U).max() < 1e-14
    assert np.abs(s1.V).max() == 0.0 and np.abs(s1.W).max() == 0.0
    # third order, not the exponential: the z^4 / 24 term is visible when |z| is large
    if abs(z) > 0.05:
        assert abs(np.exp(z) - amp) > 100 * 1e-14


@pytest.mark.parametrize("walls", [False, True])
def test_uniform_conformation_relaxes_by_the_rk3_stability_polynomial(walls):
    """Fluid at rest with a uniform Oldroyd-B conformation: div tau = 0 keeps it at
    rest, and B - I obeys dB/dt = -(B - I)/lambda exactly (Eq. SRM2, Table 1 with
    F = a = 1).  One step of Eq. rk3tau with the weights of Eq. RK multiplies B - I by
    1 + z + z^2/2 + z^3/6, z = -dt/lambda, in every cell and component."""
    ly = 2.0 if walls else 2 * np.pi
    g = oracle.Grid(8, 6, 10, 2 * np.pi, ly, 2 * np.pi, walls)
    prm = oracle.Params.from_groups('oldroyd_b', Re=2.0, Wi=0.3, beta=0.4)
    B0 = [1.7, 0.3, -0.2, 1.2, 0.1, 0.9]
    eye = [1.0, 0.0, 0.0, 1.0, 0.0, 1.0]
    s = oracle.State.rest(g)
    s.B = [np.full(g.shape, b) for b in B0]
    dt = 0.05
    s1 = oracle.rk3_step(s, dt, g, prm)
    z = -dt / prm.lam
    amp = 1.0 + z + z * z / 2.0 + z ** 3 / 6.0
    for c in range(6):
        assert np.abs(s1.B[c] - (eye[c] + amp * (B0[c] - eye[c]))).max() < 1e-15
    assert max(np.abs(a).max() for a in (s1.U, s1.V, s1.W)) == 0.0


# ---------------------------------------------------------------------------
# Saramito channel (Sec. 4.1.1 geometry, Table 1 Saramito row): plug width and
# the yielded profile of the steady pressure-driven flow


def saramito_channel_closed_form(G, mu_s, mu_p, lam, tau_y):
    """Steady yielded simple shear of the Saramito model with the velocity
    gradient du/dy = -gdot: tau_yy = 0, F tau_xy = mu_p gdot, tau_xx =
    2 lam tau_xy^2 / mu_p and F = 1 - tau_y/|tau^d|, |tau^d|^2 = tau_xy^2 +
    tau_xx^2/3.  The shear stress T = |tau_xy| parametrises everything: with the
    momentum balance mu_s gdot + T = G |y| the position of a yielded layer is
    explicit in T.  The plug edge is where gdot -> 0, |tau^d| = tau_y and T = G y0:
    (G y0)^2 = 3 mu_p^2 (-1 + sqrt(1 + 16 lam^2 tau_y^2 / (3 mu_p^2))) / (8 lam^2).
    Returns (y0, gdot(y), u(y)) with u = 0 at the walls y = +-1."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    y0 = np.sqrt(3 * mu_p ** 2 * (-1 + np.sqrt(1 + 16 * lam ** 2 * tau_y ** 2 / (3 * mu_p ** 2)))
                 / (8 * lam ** 2)) / G

    def F_of(T):
        return max(0.0, 1.0 - tau_y / np.sqrt(T ** 2 + (2 * lam * T ** 2 / mu_p) ** 2 / 3))

    def gdot(y):
        y = abs(y)
        if y <= y0:
            return 0.0
        T = brentq(lambda T: mu_s * F_of(T) * T / mu_p + T - G * y, G * y0, G * y, xtol=1e-15)
        return F_of(T) * T / mu_p

    def u(y):
        return quad(gdot, max(abs(y), y0), 1.0, epsabs=1e-13, epsrel=1e-12)[0]

    return y0, gdot, u


def test_saramito_plug_edge_closed_form_is_the_yield_root():
    """The plug-edge formula is the root of |tau^d|(T) = tau_y with tau_xx =
    2 lam T^2 / mu_p, found here by bisection; at the channel workload's values
    (G = 2/Re = 0.02, mu_p = tau_y = 0.005, lambda = 1) it gives y0 = 0.1885, and
    the Bingham limit lambda -> 0 gives tau_y / G."""
    from scipy.optimize import brentq
    for G, mu_p, lam, ty in ((0.02, 0.005, 1.0, 0.005), (1.0, 0.48, 0.8, 0.4), (3.0, 0.2, 2.5, 1.1)):
        y0, _, _ = saramito_channel_closed_form(G, 0.1, mu_p, lam, ty)
        T = brentq(lambda T: T ** 2 + (2 * lam * T ** 2 / mu_p) ** 2 / 3 - ty ** 2, 0.0, ty)
        assert abs(G * y0 - T) < 1e-12 * max(1.0, T)
    y0, _, _ = saramito_channel_closed_form(0.02, 0.005, 0.005, 1.0, 0.005)
    assert abs(y0 - 0.1885) < 5e-5
    y0, _, _ = saramito_channel_closed_form(0.02, 0.005, 0.005, 1e-3, 0.005)
    assert abs(y0 - 0.25) < 1e-5


SARAMITO_CHANNEL = dict(ny=32, Re=1.25, Wi=0.8, beta=0.4, Bi=0.5, G=1.0, T=3.0)


def saramito_channel_errors():
    """Runs the oracle's RK3 step on a thin wall-bounded channel (1 x 32 x 1, walls
    at y = +-1, body force G along x) from the closed-form steady state until the
    discrete flow is steady, and measures it against what the closed form fixes
    exactly or to O(dy^2).  mu_s, mu_p, lambda and tau_y are all different, so a
    wrong scaling of any of them shows.  Returns a dict of errors (NaN-safe: a
    diverging run gives inf)."""
    c = SARAMITO_CHANNEL
    ny, G = c['ny'], c['G']
    g = oracle.Grid(1, ny, 1, 1.0, 2.0, 1.0, True)
    prm = oracle.Params.from_groups('saramito', c['Re'], c['Wi'], c['beta'], Bi=c['Bi'])
    mu_s, mu_p, lam, ty = prm.mu_s, prm.mu_p, prm.lam, prm.tau_y
    y0, gdot, u_of = saramito_channel_closed_form(G, mu_s, mu_p, lam, ty)
    yc = g.yc()[0, :, 0]
    ua = np.array([u_of(y) for y in yc])
    # closed-form start: total shear stress -G y, tau_xx = 2 lam tau_xy^2 / mu_p
    txy = np.array([-G * y + mu_s * gdot(y) * np.sign(y) for y in yc])
    gm = mu_p / lam
    one = np.ones(g.shape)
    zero = g.zeros()
    B = [one + (2 * lam * txy ** 2 / mu_p / gm)[None, :, None], one * (txy / gm)[None, :, None], zero.copy(),
         one.copy(), zero.copy(), one.copy()]
    s = oracle.State.rest(g, U=one * ua[None, :, None])
    s.B = B
    dt = 0.9 * 2.51 / (4 * mu_s * (1 / g.dx ** 2 + 1 / g.dy ** 2 + 1 / g.dz ** 2))
    for _ in range(int(c['T'] / dt)):
        s = oracle.rk3_step(s, dt, g, prm, (G, 0.0, 0.0))
    u = s.U[0, :, 0]
    tau = [t[0, :, 0] for t in oracle.models.tau_from_B(s.B, prm)]
    F_or = np.broadcast_to(oracle.models.closure(s.B, prm)[0], g.shape)[0, :, 0]
    gd = oracle.velocity_gradient(s.U, s.V, s.W, g)[0][1][0, :, 0]
    # |tau^d| from the 3x3 stress matrix, written independently of the oracle
    M = np.zeros((ny, 3, 3))
    for k, (a, b) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        M[:, a, b] = M[:, b, a] = tau[k]
    dev = M - np.trace(M, axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
    mag = np.sqrt(0.5 * np.einsum('nij,nij->n', dev, dev))
    F_t = np.maximum(0.0, 1.0 - ty / mag)
    yielded = F_or > 0
    strong = F_t >= 0.1
    ay = np.abs(yc)
    edge_y = 0.5 * (yc[1:] + yc[:-1])
    bal = mu_s * (u[1:] - u[:-1]) / g.dy + 0.5 * (tau[1][1:] + tau[1][:-1]) + G * edge_y

    def worst(x):
        x = np.asarray(x, dtype=float)
        return float(np.max(np.abs(x))) if x.size and np.all(np.isfinite(x)) else np.inf

    return {
        # the discrete momentum balance: total shear stress = -G y at every y edge
        'force_balance': worst(bal),
        # the yield surface: unyielded cells inside y0, yielded cells outside it
        'plug_inside_y0': float(ay[~yielded].max() - y0) if np.any(~yielded) else np.inf,
        'yield_outside_y0': float(y0 - ay[yielded].min()) if np.any(yielded) else np.inf,
        'plug_cells': int(np.sum(~yielded)),
        # the oracle's F equals 1 - tau_y/|tau^d| from the stress it returns
        'F_consistent': worst((F_or - F_t)[yielded]),
        # steady yielded shear: tau_yy = 0, F tau_xy = mu_p gdot, tau_xx = 2 lam tau_xy^2 / mu_p
        'tau_yy': worst(tau[3][yielded]),
        'F_tauxy': worst((F_t * tau[1] - mu_p * gd)[strong]),
        'tau_xx': worst((tau[0] - 2 * lam * tau[1] ** 2 / mu_p)[strong]),
        # the plug moves rigidly
        'plug_gdot': worst(gd[~yielded]),
        # the velocity profile of the closed form, to O(dy^2)
        'u_rel': worst(u - ua) / ua.max(),
    }


SARAMITO_CHANNEL_TOL = {'force_balance': 5e-4, 'plug_inside_y0': 0.0, 'yield_outside_y0': 0.0,
                        'F_consistent': 1e-12, 'tau_yy': 1e-12, 'F_tauxy': 1e-3, 'tau_xx': 5e-3,
                        'plug_gdot': 5e-3, 'u_rel': 1e-2}


def saramito_channel_failures(err):
    fails = [k for k, tol in SARAMITO_CHANNEL_TOL.items() if not (err[k] <= tol)]
    if err['plug_cells'] < 6:
        fails.append('plug_cells')
    return fails


def test_saramito_channel_plug_width_and_yielded_profile():
    """Steady Saramito channel flow (Sec. 4.1.1 geometry, Table 1): the oracle's
    plug spans |y| < y0 of the closed form to within the cell layout (the edge lies
    between the last unyielded and the first yielded cell centre; the Bingham
    value tau_y/G = 0.4 here lies outside that interval), the yielded cells obey the
    steady-shear relations of the closed form, the total shear stress balances the
    body force at every edge, and u matches the closed-form profile to O(dy^2)."""
    err = saramito_channel_errors()
    assert not saramito_channel_failures(err), err


def _saramito_mag_without_half(B, prm):
    """Planted mistake: |tau^d| without the factor 1/2 of the second invariant."""
    g = prm.mu_p / prm.lam
    t = [g * (B[c] - (1.0 if c in (0, 3, 5) else 0.0)) for c in range(6)]
    tr = t[0] + t[3] + t[5]
    d = [t[c] - (tr / 3.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    mag = np.sqrt(d[0] ** 2 + d[3] ** 2 + d[5] ** 2 + 2 * (d[1] ** 2 + d[2] ** 2 + d[4] ** 2))
    F = np.where(mag > 0.0, np.maximum(0.0, 1.0 - prm.tau_y / np.where(mag > 0, mag, 1.0)), 0.0)
    return F, F


@pytest.mark.parametrize('plant', ['closure_norm', 'tau_modulus'])
def test_saramito_channel_pin_catches_planted_mistakes(plant, monkeypatch):
    """The channel pin fails when a mistake is planted in the oracle's Saramito
    closure (the second invariant without its factor 1/2) or in its stress from B
    (mu_p in place of the modulus mu_p/lambda)."""
    import oracle.models as om
    import oracle.step as ost
    if plant == 'closure_norm':
        orig = om.closure
        monkeypatch.setattr(om, 'closure', lambda B, prm: _saramito_mag_without_half(B, prm)
                            if prm.model == 'saramito' else orig(B, prm))
    else:
        orig = om.tau_from_B

        def bad(B, prm):
            if prm.model != 'saramito':
                return orig(B, prm)
            return [prm.mu_p * (B[c] - (1.0 if c in (0, 3, 5) else 0.0)) for c in range(6)]
        monkeypatch.setattr(om, 'tau_from_B', bad)
        monkeypatch.setattr(ost, 'tau_from_B', bad)
    with np.errstate(all='ignore'):
        err = saramito_channel_errors()
    assert saramito_channel_failures(err), err
