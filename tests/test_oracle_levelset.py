"""Pins for the oracle's level set, interface force and AB2 step (Secs. 3.2.1, 3.2.2)."""

import numpy as np
import pytest

import oracle
from oracle import levelset as ls
from oracle.ab2 import TwoPhase, ab2_step
from oracle.models import Params, rt_local
from paper_1803_09563_gb300 import inputs


def box(n, L=2.0):
    return oracle.Grid(n, n, n, L, L, L)


def sphere(g, c, R):
    geo = inputs.geometry(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, g.walls)
    return inputs.sphere_distance(geo, c, R)


def test_heaviside_and_delta_integrate_to_volume_and_area():
    """For a signed distance to a sphere, int(1 - H) and int(delta) have closed
    forms: the volume plus 16 pi R eps^2 (1/12 - 1/(2 pi^2)) and the area times
    (1 + eps^2 (1/3 - 2/pi^2)/R^2), from integrating the smoothed profiles
    across the shell.  The grid quadrature matches them to 1e-4."""
    g = box(48)
    R = 0.55
    phi = sphere(g, (1.0, 1.0, 1.0), R)
    eps = 1.5 * g.dx
    dv = g.dx ** 3
    vol = ((1.0 - ls.heaviside(phi, eps)).sum() * dv)
    area = ls.delta(phi, eps).sum() * dv
    vol_ref = 4.0 / 3.0 * np.pi * R ** 3 + 16.0 * np.pi * R * eps ** 2 * (1.0 / 12.0 - 0.5 / np.pi ** 2)
    area_ref = 4.0 * np.pi * (R ** 2 + eps ** 2 * (1.0 / 3.0 - 2.0 / np.pi ** 2))
    assert abs(vol - vol_ref) / vol_ref < 1e-4, (vol, vol_ref)
    assert abs(area - area_ref) / area_ref < 1e-3, (area, area_ref)
    # H is 0 deep inside, 1 far outside, 1/2 on the interface; delta = dH/dphi
    assert ls.heaviside(np.array(-1.0), eps) == 0.0 and ls.heaviside(np.array(1.0), eps) == 1.0
    assert ls.heaviside(np.array(0.0), eps) == 0.5
    x = np.linspace(-eps, eps, 101)
    num = np.gradient(ls.heaviside(x, eps), x)
    assert np.abs(num - ls.delta(x, eps))[2:-2].max() < 1e-2 / eps


def test_sphere_curvature_is_minus_two_over_r():
    """kappa = -div n (Eq. curv): -2/R on the interface of a sphere (phi > 0 outside)."""
    for n, tol in ((32, 0.05), (64, 0.02)):
        g = box(n)
        R = 0.6
        phi = sphere(g, (1.0, 1.0, 1.0), R)
        kap = ls.curvature(ls.normals(phi, g), g)
        band = np.abs(phi) < 0.5 * g.dx
        rel = np.abs(kap[band] + 2.0 / (R + phi[band])).max() * R / 2.0
        assert rel < tol, (n, rel)


def test_uniform_translation_returns_sphere():
    """Uniform velocity across one period: the zero level set returns to its start."""
    n = 32
    g = oracle.Grid(n, n, n, 2.0, 2.0, 2.0)
    phi0 = sphere(g, (1.0, 1.0, 1.0), 0.5)
    U = np.full(g.shape, 1.0)
    V = np.full(g.shape, 0.5)
    W = np.zeros(g.shape)
    phi = phi0.copy()
    steps = 80
    dt = 2.0 / steps      # one period in x, half in y
    for _ in range(steps):
        phi = ls.advect(phi, U, V, W, g, dt)
    # shifted back by (2, 1, 0): the y shift of half a period is 16 cells
    ref = np.roll(phi0, -16, axis=1)
    band = np.abs(ref) < 2 * g.dx
    assert np.abs(phi - ref)[band].max() < 0.02 * g.dx
    # the interface did not move: sign agrees away from the resolution limit
    assert np.all(np.sign(phi[np.abs(ref) > g.dx]) == np.sign(ref[np.abs(ref) > g.dx]))


def test_reinitialisation_keeps_distance_and_repairs_a_distorted_field():
    g = box(40)
    phi0 = sphere(g, (1.0, 1.0, 1.0), 0.6)
    band = np.abs(phi0) < 3 * g.dx
    # an exact signed distance is (nearly) a fixed point
    phi1 = ls.reinitialise(phi0, g, 3)
    assert np.abs(phi1 - phi0)[band].max() < 0.05 * g.dx
    # a stretched field phi0 * (2 + x) keeps its zero level set and recovers |grad| ~ 1
    x = g.xc() + 0 * phi0
    bad = phi0 * (2.0 + 0.5 * x)
    fixed = ls.reinitialise(bad, g, 20)
    gx, gy, gz = np.gradient(fixed, g.dx)
    gn = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2)
    near = np.abs(phi0) < 1.5 * g.dx
    assert np.abs(gn[near] - 1.0).mean() < 0.1
    assert np.abs(fixed - phi0)[np.abs(phi0) < 0.5 * g.dx].max() < 0.3 * g.dx


def test_ab2_coefficients_second_order_on_an_ode():
    """The AB2 weights (3/2, -1/2) with a forward-Euler first step converge at
    second order on the Oldroyd-B start-up shear closed form."""
    prm = Params.from_groups('oldroyd_b', Re=1.0, Wi=0.7, beta=0.3)
    L = [[0.0, 1.0, 0.0], [0.0] * 3, [0.0] * 3]

    def run(dt, T=1.0):
        B = [np.array(1.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
        hist = None
        for n in range(int(round(T / dt))):
            rt = rt_local(B, L, prm)
            w1, w0 = (1.0, 0.0) if n == 0 else (1.5, -0.5)
            B = [B[c] + dt * (w1 * rt[c] + (w0 * hist[c] if w0 else 0.0)) for c in range(6)]
            hist = rt
        return prm.mu_p / prm.lam * B[1]

    ref = prm.mu_p * 1.0 * (1.0 - np.exp(-1.0 / prm.lam))
    errs = [abs(run(dt) - ref) for dt in (0.02, 0.01, 0.005)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.9, errs


def test_ab2_drop_step_is_projected_and_rises():
    """A few AB2 steps of the EVP drop: divergence <= 1e-12 after each projection,
    the drop volume is kept to a few percent, and buoyancy lifts the drop."""
    n = 24
    g = oracle.Grid(n, 2 * n, n, 1.5, 3.0, 1.5)
    phi = sphere(g, (0.75, 0.9, 0.75), 0.35)
    tp = TwoPhase('saramito', Re=35.0, Wi=1.0, beta=0.5, tau_y=0.02, sigma=0.1, drho_g=1.0,
                  reinit_every=3, reinit_iters=2)
    s = oracle.State.rest(g)
    s.RT_hist, s.N_hist = None, None
    eps = tp.eps_cells * g.dx
    vol0 = (1.0 - ls.heaviside(phi, eps)).sum()
    for it in range(6):
        s, phi = ab2_step(s, phi, 2e-2, g, tp, it)
        assert np.abs(oracle.divergence(s.U, s.V, s.W, g)).max() < 1e-12
    vol = (1.0 - ls.heaviside(phi, eps)).sum()
    assert abs(vol - vol0) / vol0 < 0.05
    Hin = 1.0 - ls.heaviside(phi, eps)
    vbar = (0.5 * (s.V + oracle.at(s.V, g, 'v', j=-1)) * Hin).sum() / Hin.sum()
    assert vbar > 0.0


def variable_coefficient_matrix(g, rf):
    """div((1/rho_f) grad p) assembled independently as a sparse matrix (periodic
    x, z; y periodic or walls with no flux)."""
    import scipy.sparse as sp
    nx, ny, nz = g.nx, g.ny, g.nz
    idx = lambda i, j, k: (k * ny + j) * nx + i
    rows, cols, vals = [], [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                # faces: +x at (i), -x at (i-1), etc.; coefficient 1/rho_f / h^2
                for (di, dj, dk, h, fa) in ((1, 0, 0, g.dx, rf[0][k, j, i]), (-1, 0, 0, g.dx, rf[0][k, j, (i - 1) % nx]),
                                            (0, 1, 0, g.dy, rf[1][k, j, i] if j < ny else 0),
                                            (0, -1, 0, g.dy, rf[1][k, (j - 1) % ny, i]),
                                            (0, 0, 1, g.dz, rf[2][k, j, i]), (0, 0, -1, g.dz, rf[2][(k - 1) % nz, j, i])):
                    jj = j + dj
                    if g.walls and (jj < 0 or jj >= ny):
                        continue
                    c = idx((i + di) % nx, jj % ny, (k + dk) % nz)
                    coef = 1.0 / fa / h ** 2
                    rows += [r, r]
                    cols += [c, r]
                    vals += [coef, -coef]
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.ncells, g.ncells))


@pytest.mark.parametrize("walls", [False, True])
def test_split_projection_is_exact_and_converges_to_variable_coefficient_solution(walls):
    """Dong-Shen splitting (Eqs. poisson-LS, projection-LS): every split projection
    leaves max|div u| <= 1e-12, and iterating it with p_hat -> p^{n+1} on a fixed
    u* converges to the solution of div((1/rho) grad p) = div(u*)/dt, assembled
    here as an independent sparse matrix."""
    import scipy.sparse.linalg as spla
    from oracle.ab2 import split_projection, face_mean
    g = oracle.Grid(8, 6, 6, 2.0, 2.0, 2.0, walls)
    rng = np.random.default_rng(5)
    star = [rng.standard_normal(g.shape) for _ in range(3)]
    if walls:
        star[1][:, -1] = 0.0
    phi = sphere(g, (1.0, 0.0 if walls else 1.0, 1.0), 0.6)
    H = ls.heaviside(phi, 1.5 * g.dx)
    rho = H + 0.1 * (1.0 - H)
    dt = 0.05
    p = np.zeros(g.shape)
    # fixed point p_hat = p (contraction 1 - rho_0/rho_max = 0.9 per sweep)
    for it in range(400):
        U, V, W, pn = split_projection(star, p, p, rho, dt, g, 0.1)
        if it % 50 == 0:
            assert np.abs(oracle.divergence(U, V, W, g)).max() < 1e-12 * max(1.0, np.abs(star[0]).max() / g.dx)
        p = pn
    A = variable_coefficient_matrix(g, face_mean(rho, g))
    b = oracle.divergence(*star, g).ravel() / dt
    A2 = A.tolil()
    A2[0, :] = 0.0
    A2[0, 0] = 1.0
    b[0] = p.ravel()[0]
    ref = spla.spsolve(A2.tocsr(), b).reshape(g.shape)
    assert np.abs(p - ref).max() < 1e-8 * np.abs(ref).max()


def test_split_projection_uniform_density_is_the_standard_projection():
    from oracle.ab2 import split_projection
    g = oracle.Grid(8, 6, 6, 2.0, 2.0, 2.0)
    rng = np.random.default_rng(6)
    star = [rng.standard_normal(g.shape) for _ in range(3)]
    p0 = rng.standard_normal(g.shape)
    U, V, W, p = split_projection(star, p0, p0, np.ones(g.shape), 0.05, g, 1.0)
    U2, V2, W2, psi = oracle.project(star[0], star[1], star[2], g, 0.05)
    for a, b in ((U, U2), (V, V2), (W, W2), (p, psi)):
        assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(b).max())


def test_light_drop_rises_with_density_contrast():
    """k_rho = 0.1 drop under gravity (Sec. 4.2.3 rising-drop setting): projected
    steps, the drop's mean vertical velocity turns positive."""
    n = 16
    g = oracle.Grid(n, 2 * n, n, 1.5, 3.0, 1.5)
    phi = sphere(g, (0.75, 0.9, 0.75), 0.35)
    tp = TwoPhase('oldroyd_b', Re=35.0, Wi=1.0, beta=0.5, tau_y=0.0, sigma=0.1, drho_g=0.0,
                  reinit_every=0, rho_ratio=0.1, gravity=1.0)
    s = oracle.State.rest(g)
    for it in range(5):
        s, phi = ab2_step(s, phi, 1e-2, g, tp, it)
        assert np.abs(oracle.divergence(s.U, s.V, s.W, g)).max() < 1e-11
    Hin = 1.0 - ls.heaviside(phi, 1.5 * g.dx)
    vbar = (0.5 * (s.V + oracle.at(s.V, g, 'v', j=-1)) * Hin).sum() / Hin.sum()
    assert vbar > 0.0


def test_mass_correction_undoes_a_uniform_shift():
    """Reading 17: for an exact signed distance phi of a sphere, the correction of
    phi + 0.013 back to the volume of phi returns phi (the smoothed volume is a
    strictly decreasing function of the shift, so the Newton root is -0.013)."""
    n, L = 32, 1.0
    g = oracle.Grid(n, n, n, L, L, L)
    geo = inputs.geometry(n, n, n, L, L, L)
    phi = inputs.sphere_distance(geo, (0.5, 0.47, 0.52), 0.23)
    eps = 1.5 * g.dx
    v0 = ls.drop_volume(phi, g, eps)
    out = ls.mass_correct(phi + 0.013, g, eps, v0, iters=6)
    assert np.abs(out - phi).max() < 1e-12
    assert abs(ls.drop_volume(out, g, eps) - v0) < 1e-13 * v0
    # zero iterations and a field already at v0 leave phi unchanged
    np.testing.assert_array_equal(ls.mass_correct(phi, g, eps, v0, iters=0), phi)
    assert np.abs(ls.mass_correct(phi, g, eps, v0, iters=3) - phi).max() == 0.0


def test_mass_correction_keeps_the_drop_volume_over_ab2_steps():
    """With the correction on, the smoothed drop volume after every AB2 step equals
    the initial one (to the Newton tolerance); without it, advection and
    re-distancing change it."""
    n = 16
    g = oracle.Grid(n, 2 * n, n, 1.5, 3.0, 1.5)
    geo = inputs.geometry(n, 2 * n, n, 1.5, 3.0, 1.5)
    phi0 = inputs.sphere_distance(geo, (0.75, 0.9, 0.75), 0.35)
    eps = 1.5 * g.dx
    v0 = ls.drop_volume(phi0, g, eps)
    drift = {}
    for iters in (0, 4):
        tp = TwoPhase('saramito', Re=35.0, Wi=1.0, beta=0.5, tau_y=0.02, sigma=0.1, drho_g=1.0,
                      reinit_every=2, reinit_iters=2, mass_iters=iters)
        st, phi = oracle.State.rest(g), phi0.copy()
        for it in range(4):
            st, phi = ab2_step(st, phi, 2e-2, g, tp, it)
        drift[iters] = abs(ls.drop_volume(phi, g, eps) - v0) / v0
    assert drift[4] < 1e-12 and drift[0] > 1e-6, drift


def test_csf_force_of_a_drop_at_rest_gives_the_laplace_jump():
    """Laplace's law for the CSF force sigma kappa delta(phi) n (Eq. fLS): the
    pressure that balances it (lap p = div F, the projection of F) is uniform inside
    and outside a spherical drop and higher inside by 2 sigma / R.  This fixes the
    sign of kappa and n and the magnitude of delta together."""
    n, L, R, sigma = 32, 2.0, 0.5, 0.1
    g = box(n, L)
    phi = sphere(g, (1.0, 1.0, 1.0), R)
    eps = 1.5 * g.dx
    F = ls.centres_to_faces(ls.interface_force_centres(phi, g, sigma, eps, 0.0), g)
    p = oracle.solve_poisson(oracle.divergence(*F, g), g)
    inside, outside = phi < -3 * eps, phi > 3 * eps
    jump = p[inside].mean() - p[outside].mean()
    assert abs(jump / (2.0 * sigma / R) - 1.0) < 0.01
    assert p[inside].std() < 1e-3 * jump and p[outside].std() < 1e-3 * jump


def test_buoyancy_is_mean_free_and_lifts_the_drop():
    """Boussinesq buoyancy (1 - H) drho_g e_y minus its domain mean: zero net force,
    x and z parts zero, and a difference of exactly drho_g between the drop
    (phi < -eps, 1 - H = 1) and the outer fluid (phi > eps)."""
    g = box(24)
    phi = sphere(g, (1.0, 0.8, 1.0), 0.45)
    eps = 1.5 * g.dx
    fx, fy, fz = ls.interface_force_centres(phi, g, 0.0, eps, 0.7)
    assert np.abs(fx).max() == 0.0 and np.abs(fz).max() == 0.0
    assert abs(fy.sum()) < 1e-12 * np.abs(fy).sum()
    inside, outside = phi < -eps, phi > eps
    assert np.allclose(fy[inside], fy[inside][0]) and np.allclose(fy[outside], fy[outside][0])
    assert abs(fy[inside][0] - fy[outside][0] - 0.7) < 1e-14
    assert fy[inside][0] > 0.0


def _cube_maps():
    """Axis swaps and mirrors of a periodic cube as maps of (face vector, centre
    scalar, centre vector) fields, [z][y][x] storage."""
    AX = (2, 1, 0)
    maps = []
    for a, b in ((0, 1), (1, 2), (0, 2)):
        s = [0, 1, 2]
        s[a], s[b] = b, a
        sw = (lambda a_, b_: (lambda f: np.swapaxes(f, AX[a_], AX[b_]).copy()))(a, b)
        vec = (lambda sw_, s_: (lambda v: [sw_(v[s_[q]]) for q in range(3)]))(sw, s)
        maps.append(('swap%d%d' % (a, b), vec, sw, vec))
    for a in range(3):
        ax = AX[a]
        rc = (lambda ax_: (lambda f: np.flip(f, ax_).copy()))(ax)
        rf = (lambda ax_: (lambda f: -np.roll(np.flip(f, ax_), -1, axis=ax_)))(ax)
        fvec = (lambda a_, rc_, rf_: (lambda v: [rf_(v[q]) if q == a_ else rc_(v[q]) for q in range(3)]))(a, rc, rf)
        cvec = (lambda a_, rc_: (lambda v: [-rc_(v[q]) if q == a_ else rc_(v[q]) for q in range(3)]))(a, rc)
        maps.append(('mirror%d' % a, fvec, rc, cvec))
    return maps


@pytest.mark.parametrize("name,fvec,cen,cvec", _cube_maps(), ids=[m[0] for m in _cube_maps()])
def test_level_set_operators_commute_with_the_cube_symmetries(name, fvec, cen, cvec):
    """Level-set advection (WENO5, Eq. ls-adv), the re-distancing right-hand side
    (Godunov upwinding, Eq. reinit), the normals and curvature and the CSF force
    (Eqs. normal, curv, fLS): each maps transformed inputs to the transformed
    result.  The drop is off-centre, the velocity random, so no symmetry of the
    data hides a one-direction typo."""
    n, L = 16, 2.0
    g = box(n, L)
    geo = inputs.geometry(n, n, n, L, L, L)
    phi = sphere(g, (0.9, 1.1, 1.05), 0.45) * (1.0 + 0.2 * np.sin(np.pi * g.xc()) * np.cos(np.pi * g.zc()))
    vel = list(inputs.scale_max(*inputs.random_solenoidal(geo, 7, 3), 1.0))
    eps = 1.5 * g.dx
    ref = ls.advection_rhs(phi, *vel, g)
    got = ls.advection_rhs(cen(phi), *fvec(vel), g)
    assert np.abs(got - cen(ref)).max() < 1e-13 * np.abs(ref).max()
    phi0 = sphere(g, (0.9, 1.1, 1.05), 0.45)
    ref = ls.reinit_rhs(phi, phi0, g)
    got = ls.reinit_rhs(cen(phi), cen(phi0), g)
    assert np.abs(got - cen(ref)).max() < 1e-13 * np.abs(ref).max()
    ref = ls.curvature(ls.normals(phi, g), g)
    got = ls.curvature(ls.normals(cen(phi), g), g)
    assert np.abs(got - cen(ref)).max() < 1e-12 * np.abs(ref).max()
    ref = ls.interface_force_centres(phi, g, 0.1, eps, 0.0)
    got = ls.interface_force_centres(cen(phi), g, 0.1, eps, 0.0)
    scale = max(np.abs(r).max() for r in ref)
    for a, b in zip(got, cvec(list(ref))):
        assert np.abs(a - b).max() < 1e-12 * scale


def test_ab2_shear_mode_follows_the_ab2_recurrence():
    """One fluid everywhere (phi = 5, H = 1, no interface force, zero mean-free
    buoyancy; beta = 1 so tau = 0): a shear mode u = sin(m y) e_x decays under
    u' = -nu lambda u with lambda the discrete Laplacian eigenvalue, and the AB2 step
    of Eqs. ab2 / ru (forward Euler first, Reading 11; the variable-viscosity form
    with the mixture viscosity) gives exactly u^1 = (1 + z) u^0 and
    u^{n+1} = u^n + z (3/2 u^n - 1/2 u^{n-1}), z = -nu lambda dt."""
    g = oracle.Grid(8, 16, 6, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    m, dt = 2, 0.01
    U = np.broadcast_to(np.sin(m * g.yc()), g.shape).copy()
    tp = TwoPhase('oldroyd_b', Re=0.5, Wi=1.0, beta=1.0, tau_y=0.0, sigma=0.1, drho_g=1.0, reinit_every=0)
    z = -(tp.beta / tp.Re) * (2.0 - 2.0 * np.cos(m * g.dy)) / g.dy ** 2 * dt
    s, phi = oracle.State.rest(g, U), np.full(g.shape, 5.0)
    ref = [U, (1.0 + z) * U]
    for n in range(4):
        s, phi = ab2_step(s, phi, dt, g, tp, n)
        if n >= 1:
            ref.append(ref[-1] + z * (1.5 * ref[-1] - 0.5 * ref[-2]))
        assert np.abs(s.U - ref[n + 1]).max() < 1e-14
        assert np.abs(s.V).max() == 0.0 and np.abs(s.W).max() == 0.0
