"""Pins for the oracle's staggered-grid operators: centre velocity, velocity
gradient (Reading 5), stress-RHS assembly (Eqs. rt / RK-rt) and the momentum
operators (Eq. NS-num1)."""

import numpy as np
import pytest

import oracle
from oracle.models import rt_local, Params
from paper_1803_09563_gb300 import inputs


def box(nx=12, ny=10, nz=8, walls=False):
    ly = 2.0 if walls else 2 * np.pi
    return oracle.Grid(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)


def test_velocity_gradient_closed_forms():
    """u = (sin y + sin z + sin x, ...): every entry L_ij = du_i/dx_j of the
    discrete gradient matches the closed form of its stencil -- a face difference
    for i = j (factor sin(h/2)/(h/2)), a central difference of centre values for
    i != j (factor sin(h)/h)."""
    g = box(16, 12, 10)
    xc, yc, zc, xf, yf, zf = g.xc(), g.yc(), g.zc(), g.xf(), g.yf(), g.zf()
    a = np.array([[1.0, 2.0, 3.0], [0.5, 1.5, -1.0], [-2.0, 0.7, 1.1]])
    # u_i = a_ix sin(x) + a_iy sin(y) + a_iz sin(z), each at the face of component i
    U = a[0, 0] * np.sin(xf) + a[0, 1] * np.sin(yc) + a[0, 2] * np.sin(zc) + 0 * xf * yc * zc
    V = a[1, 0] * np.sin(xc) + a[1, 1] * np.sin(yf) + a[1, 2] * np.sin(zc) + 0 * xc * yf * zc
    W = a[2, 0] * np.sin(xc) + a[2, 1] * np.sin(yc) + a[2, 2] * np.sin(zf) + 0 * xc * yc * zf
    L = oracle.velocity_gradient(U, V, W, g)
    h = (g.dx, g.dy, g.dz)
    cc = (xc, yc, zc)
    for i in range(3):
        for j in range(3):
            fac = np.sin(h[j] / 2) / (h[j] / 2) if i == j else np.sin(h[j]) / h[j]
            ref = a[i, j] * np.cos(cc[j]) * fac
            np.testing.assert_allclose(L[i][j], np.broadcast_to(ref, g.shape), atol=1e-12)


def test_stress_rhs_uses_L_not_its_transpose():
    """With a uniform B the advection vanishes exactly and the assembled RT equals
    the pointwise source with the closed-form gradient; a simple shear u = sin(y)
    must load tau_xx (upper-convected), not tau_yy."""
    g = box(8, 16, 6)
    U = np.broadcast_to(np.sin(g.yc()), g.shape).copy()
    V, W = g.zeros(), g.zeros()
    prm = Params.from_groups('oldroyd_b', Re=1.0, Wi=1.0, beta=0.5)
    B0 = [1.0, 0.2, 0.0, 1.0, 0.0, 1.0]
    B = [np.full(g.shape, b) for b in B0]
    rt = oracle.stress_rhs(U, V, W, B, g, prm)
    Lxy = np.cos(g.yc()) * np.sin(g.dy) / g.dy
    # d Bxx/dt = 2 Lxy Bxy ; d Byy/dt = 0 ; d Bxy/dt = Lxy Byy - Bxy/lam
    np.testing.assert_allclose(rt[0], np.broadcast_to(2 * Lxy * 0.2, g.shape), atol=1e-13)
    np.testing.assert_allclose(rt[3], 0.0, atol=1e-14)
    np.testing.assert_allclose(rt[1], np.broadcast_to(Lxy * 1.0 - 0.2, g.shape), atol=1e-13)


def _translate_one_period(axis, n):
    shape = {'x': (n, 4, 4), 'y': (4, n, 4), 'z': (4, 4, n)}[axis]
    g = oracle.Grid(*shape, 2 * np.pi, 2 * np.pi, 2 * np.pi)
    c = -1.0 if axis == 'y' else 1.0
    U, V, W = g.zeros(), g.zeros(), g.zeros()
    {'x': U, 'y': V, 'z': W}[axis][...] = c
    s = {'x': g.xc(), 'y': g.yc(), 'z': g.zc()}[axis]
    prm = Params('oldroyd_b', mu_s=0.0, mu_p=0.0, lam=1e30)
    B = [np.ones(g.shape) if d else np.zeros(g.shape) for d in (1, 0, 0, 1, 0, 1)]
    B[0] = np.broadcast_to(1.0 + 0.1 * np.sin(s), g.shape).copy()
    B0 = B[0].copy()
    nsteps = 5 * n
    dt = 2 * np.pi / nsteps
    hist = None
    for _ in range(nsteps):
        for k in range(3):
            rt = oracle.stress_rhs(U, V, W, B, g, prm)
            B = [B[q] + dt * (oracle.RK3_ZETA[k] * rt[q]
                              + (oracle.RK3_XI[k] * hist[q] if k else 0.0)) for q in range(6)]
            hist = rt
    assert np.abs(B[3] - 1.0).max() == 0.0
    return np.abs(B[0] - B0).max()


@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_pure_advection_translates_and_returns(axis):
    """Uniform velocity along one axis, B_xx = 1 + 0.1 sin(s) and no relaxation
    (lambda huge): one period of the RK3-WENO5 update returns B_xx to its start.
    The error falls at least 8x per refinement (CFL fixed) -- a downwind
    (unstable) or low-order scheme fails this."""
    e32 = _translate_one_period(axis, 32)
    e64 = _translate_one_period(axis, 64)
    assert e32 < 5e-5 and e64 < e32 / 8.0, (e32, e64)


def test_momentum_advection_of_uniform_flow_is_zero_and_laplacian_exact_on_modes():
    g = box(12, 10, 8)
    U = np.full(g.shape, 0.7)
    V = np.full(g.shape, -0.3)
    W = np.full(g.shape, 0.2)
    A = oracle.advection(U, V, W, g)
    for a in A:
        assert np.abs(a).max() < 1e-14
    # Laplacian of sin(2x) at x-faces: -(2 - 2cos(2h))/h^2 sin(2x)
    F = np.broadcast_to(np.sin(2 * g.xf()), g.shape).copy()
    lap = oracle.laplacian(F, g, 'u')
    ref = -(2 - 2 * np.cos(2 * g.dx)) / g.dx ** 2 * F
    np.testing.assert_allclose(lap, ref, atol=1e-12)


def test_advection_matches_conservative_form_for_a_shear_wave():
    """u = sin(y) e_x (divergence free, steady Euler solution): div(uu) = 0 in x and y."""
    g = box(8, 16, 6)
    U = np.broadcast_to(np.sin(g.yc()), g.shape).copy()
    A = oracle.advection(U, g.zeros(), g.zeros(), g)
    for a in A:
        assert np.abs(a).max() < 1e-14


def test_full_viscous_form_reduces_to_laplacian_for_uniform_mu():
    """div[mu(grad u + grad u^T)] with a uniform mu array equals mu lap(u) for a
    discretely divergence-free u (periodic and walls)."""
    for walls in (False, True):
        geo = inputs.geometry(12, 10, 8, 2 * np.pi, 2.0 if walls else 2 * np.pi, 2 * np.pi, walls)
        g = oracle.Grid(12, 10, 8, geo['lx'], geo['ly'], geo['lz'], walls)
        U, V, W = inputs.random_solenoidal(geo, 4, 3)
        mu = np.full(g.shape, 0.37)
        full = oracle.momentum.viscous(U, V, W, g, mu)
        lap = oracle.momentum.viscous(U, V, W, g, 0.37)
        for f, l in zip(full, lap):
            if walls:
                f, l = f[:, :-1], l[:, :-1]   # top wall faces are not updated
            np.testing.assert_allclose(f, l, atol=1e-10 * np.abs(l).max())


def test_div_tau_of_uniform_stress_is_zero_and_linear_stress_exact():
    g = box(10, 12, 8)
    tau = [np.full(g.shape, v) for v in (1.0, 2.0, 3.0, 4.0, 5.0, 6.0)]
    for f in oracle.div_tau(tau, g):
        assert np.abs(f).max() < 1e-14
    # tau_xy = sin(y) only: div tau = (d/dy tau_xy, d/dx tau_xy, 0) -> x-face gets
    # the y-difference of the 4-point edge averages, i.e. cos(y) sin(dy)/dy
    tau = [g.zeros() for _ in range(6)]
    tau[1] = np.broadcast_to(np.sin(g.yc()), g.shape).copy()
    fx, fy, fz = oracle.div_tau(tau, g)
    np.testing.assert_allclose(fx, np.broadcast_to(np.cos(g.yc()) * np.sin(g.dy) / g.dy, g.shape), atol=1e-12)
    assert np.abs(fy).max() < 1e-14 and np.abs(fz).max() < 1e-14


def test_wall_ghost_rules():
    g = box(6, 8, 4, walls=True)
    a = np.random.default_rng(0).standard_normal(g.shape)
    np.testing.assert_array_equal(oracle.at(a, g, 'c', j=-2)[:, 0], a[:, 0])
    np.testing.assert_array_equal(oracle.at(a, g, 'u', j=-1)[:, 0], -a[:, 0])
    np.testing.assert_array_equal(oracle.at(a, g, 'u', j=1)[:, -1], -a[:, -1])
    np.testing.assert_array_equal(oracle.at(a, g, 'v', j=-1)[:, 0], 0.0)
    np.testing.assert_array_equal(oracle.at(a, g, 'c', j=3)[:, -1], a[:, -1])


def solenoidal_case(walls, seed=5, shape=(12, 10, 14)):
    nx, ny, nz = shape
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, 2.0 if walls else 2 * np.pi, 2 * np.pi, walls)
    g = oracle.Grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls)
    U, V, W = inputs.random_solenoidal(geo, seed, 3)
    if walls:
        U = U + inputs.poiseuille(geo)[0]
    return geo, g, U, V, W


@pytest.mark.parametrize("walls", [False, True])
def test_advection_conserves_kinetic_energy_of_solenoidal_fields(walls):
    """The divergence form of div(uu) on the staggered grid with central averages
    (Sec. 3) is energy-conserving when the discrete continuity equation holds:
    sum over the faces of u.div(uu) = 0 for a discretely divergence-free field
    (periodic, or with no-penetration walls).  Every term of the three face
    components enters this sum, so a wrong neighbour, sign or spacing in any of
    them leaves a residual of order one."""
    geo, g, U, V, W = solenoidal_case(walls)
    assert np.abs(oracle.divergence(U, V, W, g)).max() < 1e-12
    A = oracle.advection(U, V, W, g)
    terms = [U * A[0], V * A[1], W * A[2]]
    total = sum(t.sum() for t in terms)
    scale = sum(np.abs(t).sum() for t in terms)
    assert abs(total) < 1e-13 * scale


@pytest.mark.parametrize("walls", [False, True])
def test_div_tau_is_minus_the_adjoint_of_the_velocity_gradient(walls):
    """Summation by parts on the staggered grid: for any symmetric centre stress tau,
    sum over the faces of u.div(tau) = -sum over the cells of L:tau, with div(tau)
    from the edge averages of Reading 5 and L from the centre velocity gradient of
    Reading 5 (periodic, or no-slip walls with their ghost rules).  It ties the two
    discretisations to each other: a wrong sign, neighbour or spacing in either
    breaks it (a transposed L does not, tau being symmetric; that case has its own
    pin above)."""
    geo, g, U, V, W = solenoidal_case(walls)
    B = inputs.random_conformation(geo, 3, amp=0.5)
    tau = [b - (1.0 if c in (0, 3, 5) else 0.0) for c, b in enumerate(B)]
    f = oracle.div_tau(tau, g)
    lhs = (U * f[0]).sum() + (V * f[1]).sum() + (W * f[2]).sum()
    L = oracle.velocity_gradient(U, V, W, g)
    comp = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    rhs = -sum((L[i][j] * tau[comp[(min(i, j), max(i, j))]]).sum() for i in range(3) for j in range(3))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("walls", [False, True])
def test_variable_viscosity_form_is_symmetric_and_dissipative(walls):
    """div[mu(grad u + grad u^T)] in divergence form with centre normal stresses and
    edge shear stresses (Sec. 3.2.1 mixture viscosity): the bilinear form
    sum a.V(b) is symmetric and sum a.V(a) < 0 for any positive mu field, periodic
    or with no-slip walls (wall faces of v held at zero)."""
    g = box(12, 10, 14, walls)
    rng = np.random.default_rng(1)
    a = [rng.standard_normal(g.shape) for _ in range(3)]
    b = [rng.standard_normal(g.shape) for _ in range(3)]
    if walls:
        a[1][:, -1] = 0.0
        b[1][:, -1] = 0.0
    mu = 0.3 + 0.2 * rng.random(g.shape)
    Va = oracle.momentum.viscous(*a, g, mu)
    Vb = oracle.momentum.viscous(*b, g, mu)
    ab = sum((a[q] * Vb[q]).sum() for q in range(3))
    ba = sum((b[q] * Va[q]).sum() for q in range(3))
    assert abs(ab - ba) < 1e-13 * abs(ab)
    assert sum((a[q] * Va[q]).sum() for q in range(3)) < 0.0


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_variable_viscosity_one_dimensional_fluxes(q, d):
    """Brute force on a periodic box: velocity component q and the viscosity vary
    along direction d only.  The form reduces to a 1-D flux difference, written
    out here cell by cell: for d != q the shear flux mu_e (f[n+1] - f[n]) / h with
    the edge viscosity mu_e = (m[n] + m[n+1]) / 2; for d == q the normal flux
    2 m[n+1] (f[n+1] - f[n]) / h with the viscosity of the centre between the two
    faces.  The other two components vanish."""
    shape = [6, 8, 10]                       # x, y, z
    g = box(*shape)
    h = (g.dx, g.dy, g.dz)[d]
    n = shape[d]
    rng = np.random.default_rng(10 * q + d)
    f = rng.standard_normal(n)
    m = 0.5 + rng.random(n)

    def along(v):
        s = [1, 1, 1]
        s[d] = n
        return np.broadcast_to(np.asarray(v).reshape(s[::-1]), g.shape).copy()

    vel = [g.zeros(), g.zeros(), g.zeros()]
    vel[q] = along(f)
    out = oracle.momentum.viscous(*vel, g, along(m))
    exp = np.zeros(n)
    for i in range(n):
        ip, im = (i + 1) % n, (i - 1) % n
        if d != q:
            up = 0.5 * (m[i] + m[ip]) * (f[ip] - f[i]) / h
            lo = 0.5 * (m[im] + m[i]) * (f[i] - f[im]) / h
        else:
            up = 2.0 * m[ip] * (f[ip] - f[i]) / h
            lo = 2.0 * m[i] * (f[i] - f[im]) / h
        exp[i] = (up - lo) / h
    np.testing.assert_allclose(out[q], along(exp), rtol=0, atol=1e-12 * np.abs(exp).max())
    for r in range(3):
        if r != q:
            assert np.abs(out[r]).max() < 1e-12 * np.abs(exp).max()


@pytest.mark.parametrize("walls", [False, True])
def test_grad_p_is_minus_the_adjoint_of_the_divergence(walls):
    """Summation by parts between the face gradient of a centre field and the centre
    divergence of a face field (Eqs. NS-num2/3): sum u.grad p = -sum p div u for any
    p and any u (wall faces of v at zero; the pressure's zero-gradient wall ghost
    makes its wall-face gradient vanish)."""
    g = box(12, 10, 14, walls)
    rng = np.random.default_rng(2)
    u = [rng.standard_normal(g.shape) for _ in range(3)]
    if walls:
        u[1][:, -1] = 0.0
    p = rng.standard_normal(g.shape)
    gp = oracle.grad_p(p, g)
    lhs = sum((u[q] * gp[q]).sum() for q in range(3))
    rhs = -(p * oracle.divergence(*u, g)).sum()
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("walls", [False, True])
def test_laplacian_is_symmetric_and_negative(walls):
    """The uniform-viscosity Laplacian of the three face components (with the no-slip
    ghosts of u, w and the zero wall face of v) is a symmetric, negative definite
    operator: sum a.lap(b) = sum b.lap(a), sum a.lap(a) < 0."""
    g = box(12, 10, 14, walls)
    rng = np.random.default_rng(3)
    a = [rng.standard_normal(g.shape) for _ in range(3)]
    b = [rng.standard_normal(g.shape) for _ in range(3)]
    if walls:
        a[1][:, -1] = 0.0
        b[1][:, -1] = 0.0
    La = oracle.momentum.viscous(*a, g, 0.3)
    Lb = oracle.momentum.viscous(*b, g, 0.3)
    ab = sum((a[q] * Lb[q]).sum() for q in range(3))
    ba = sum((b[q] * La[q]).sum() for q in range(3))
    assert abs(ab - ba) < 1e-13 * abs(ab)
    assert sum((a[q] * La[q]).sum() for q in range(3)) < 0.0


# ---- discrete symmetries of the periodic staggered cube: an axis swap or a mirror
# maps the grid onto itself, so every operator must commute with it.  Array axis
# of direction d (x 0, y 1, z 2) in [z][y][x] storage:
_AX = (2, 1, 0)
_COMP = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}


def _comp(i, j):
    return _COMP[(min(i, j), max(i, j))]


def _swap(a, b):
    """(vector map, tensor map) of the swap of directions a and b."""
    s = [0, 1, 2]
    s[a], s[b] = b, a
    sw = lambda f: np.swapaxes(f, _AX[a], _AX[b]).copy()
    vec = lambda v: [sw(v[s[q]]) for q in range(3)]
    ten = lambda t: [sw(t[_comp(s[i], s[j])]) for (i, j) in _COMP]
    return vec, ten, sw


def _mirror(a):
    """(vector map, tensor map, centre map) of the reflection x_a -> -x_a: centre
    values and the other components reverse along a; the a-face component also
    changes sign and moves from face i+1/2 to face n-1-i-1/2; tensor components
    with one index a change sign."""
    ax = _AX[a]
    rc = lambda f: np.flip(f, ax).copy()
    rf = lambda f: -np.roll(np.flip(f, ax), -1, axis=ax)
    vec = lambda v: [rf(v[q]) if q == a else rc(v[q]) for q in range(3)]
    ten = lambda t: [(-1.0 if (i == a) != (j == a) else 1.0) * rc(t[_comp(i, j)]) for (i, j) in _COMP]
    return vec, ten, rc


def _sym_case():
    n, L = 12, 2 * np.pi
    geo = inputs.geometry(n, n, n, L, L, L)
    g = oracle.Grid(n, n, n, L, L, L)
    vel = list(inputs.scale_max(*inputs.random_solenoidal(geo, 5, 3), 1.0))
    B = inputs.spd_conformation(geo, 3, 0.5, scale=2.0)
    mu = 0.3 + 0.2 * np.random.default_rng(4).random(g.shape)
    return g, vel, B, mu


def _maps():
    out = []
    for a, b in ((0, 1), (1, 2), (0, 2)):
        out.append(('swap%d%d' % (a, b),) + _swap(a, b))
    for a in range(3):
        out.append(('mirror%d' % a,) + _mirror(a))
    return out


@pytest.mark.parametrize("name,vec,ten,cen", _maps(), ids=[m[0] for m in _maps()])
@pytest.mark.parametrize("model,extra", [('saramito', {'Bi': 0.4}), ('fene_p', {'L2': 30.0}), ('oldroyd_b', {})])
def test_stress_rhs_commutes_with_the_cube_symmetries(name, vec, ten, cen, model, extra):
    """Stress RHS (Eq. rt: WENO5 advection, upper-convected terms, Table 1 closure):
    RT(S u, S B) = S RT(u, B) for the axis swaps and mirrors S of the cube.  A typo
    confined to one direction's stencil, or to the upwind side of a negative
    velocity, breaks it."""
    g, vel, B, _ = _sym_case()
    prm = oracle.Params.from_groups(model, Re=2.0, Wi=0.8, beta=0.4, **extra)
    R = oracle.stress_rhs(*vel, B, g, prm)
    Rs = oracle.stress_rhs(*vec(vel), ten(B), g, prm)
    scale = max(np.abs(r).max() for r in R)
    for got, ref in zip(Rs, ten(R)):
        assert np.abs(got - ref).max() < 1e-13 * scale


@pytest.mark.parametrize("name,vec,ten,cen", _maps(), ids=[m[0] for m in _maps()])
def test_momentum_operators_commute_with_the_cube_symmetries(name, vec, ten, cen):
    """Advection, the uniform and the variable-viscosity viscous forms, and div tau:
    each maps S-transformed inputs to the S-transformed result."""
    g, vel, B, mu = _sym_case()
    tau = [b - (1.0 if c in (0, 3, 5) else 0.0) for c, b in enumerate(B)]
    pairs = [
        (oracle.momentum_rhs_n(*vel, g, 0.3), oracle.momentum_rhs_n(*vec(vel), g, 0.3)),
        (oracle.momentum.viscous(*vel, g, mu), oracle.momentum.viscous(*vec(vel), g, cen(mu))),
        (oracle.div_tau(tau, g), oracle.div_tau(ten(tau), g)),
    ]
    for ref, got in pairs:
        scale = max(np.abs(r).max() for r in ref)
        for a, b in zip(got, vec(list(ref))):
            assert np.abs(a - b).max() < 1e-13 * scale
