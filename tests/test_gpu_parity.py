"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, row by row:
S1+S2 stress RHS, S4-S7 Poisson solve, S8 projection, whole RK3 substeps and steps.

Relative error of a field = max|gpu - oracle| / max(max|oracle|, 1e-300).
Tolerances: FP64 path 1e-10 (whole steps) / 1e-12 (single operators);
FP32 path 1e-5 per step from the same FP64 state rounded to FP32.
"""

import numpy as np
import pytest

import oracle
from paper_1803_09563_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(got, ref):
    return float(np.abs(np.asarray(got, dtype=np.float64) - ref).max() / max(np.abs(ref).max(), 1e-300))


# (nx, ny, nz, walls): several tiles of 32x8 plus ragged tails, both boundary types
SHAPES = [(48, 24, 18, False), (36, 20, 16, True), (32, 32, 32, False), (64, 12, 24, True)]
MODELS = [('oldroyd_b', {}), ('fene_p', {'L2': 60.0}), ('saramito', {'Bi': 0.4}), ('neo_hookean', {})]


def setup_case(evp, shape, model, extra, precision, seed=3, re=2.0, dpdx=0.0):
    nx, ny, nz, walls = shape
    ly = 2.0 if walls else 2 * np.pi
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, seed, 3), 1.0)
    if walls:
        U = U + inputs.poiseuille(geo)[0]
    B = inputs.random_conformation(geo, seed + 1, amp=0.3)
    p = np.random.default_rng(seed + 2).standard_normal((nz, ny, nx)) * 0.1
    g = oracle.Grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls)
    prm_o = oracle.Params.from_groups(model, Re=re, Wi=0.8, beta=0.4, **extra)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls), model,
                         evp.make_params(Re=re, Wi=0.8, beta=0.4, precision=precision, dpdx=dpdx, **extra))
    sim.set_state(U, V, W, p, B)
    st = oracle.State.rest(g, U, V, W)
    st.p = p.copy()
    st.B = [b.copy() for b in B]
    if precision == evp.EVP_FP32:
        # the oracle starts from exactly the FP32-rounded state the GPU holds
        rd = lambda a: a.astype(np.float32).astype(np.float64)
        st.U, st.V, st.W, st.p = rd(st.U), rd(st.V), rd(st.W), rd(st.p)
        st.B = [rd(b) for b in st.B]
    if walls:
        st.V[:, -1] = 0.0
    return sim, st, g, prm_o


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("model,extra", MODELS)
def test_stress_rhs_fp64(evp, shape, model, extra):
    import torch
    sim, st, g, prm = setup_case(evp, shape, model, extra, evp.EVP_FP64)
    out = torch.empty((6,) + sim.shape, dtype=torch.float64, device='cuda')
    evp.evp_stress_rhs(sim.handle, out)
    sim.sync()
    ref = oracle.stress_rhs(st.U, st.V, st.W, st.B, g, prm)
    for c in range(6):
        assert rel(out[c].cpu().numpy(), ref[c]) < 1e-12, (c, rel(out[c].cpu().numpy(), ref[c]))


@pytest.mark.parametrize("shape", SHAPES)
def test_stress_rhs_fp32(evp, shape):
    import torch
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, evp.EVP_FP32)
    out = torch.empty((6,) + sim.shape, dtype=torch.float32, device='cuda')
    evp.evp_stress_rhs(sim.handle, out)
    sim.sync()
    ref = oracle.stress_rhs(st.U, st.V, st.W, st.B, g, prm)
    for c in range(6):
        assert rel(out[c].cpu().numpy(), ref[c]) < 1e-5


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_poisson_solve(evp, shape, prec, tol):
    import torch
    nx, ny, nz, walls = shape
    sim, st, g, prm = setup_case(evp, shape, 'oldroyd_b', {}, prec)
    rng = np.random.default_rng(9)
    r = rng.standard_normal((nz, ny, nx))
    r -= r.mean()
    if prec == 1:
        r = r.astype(np.float32).astype(np.float64)
    dt = torch.float32 if prec else torch.float64
    rd = torch.tensor(r, dtype=dt, device='cuda')
    psi = torch.empty_like(rd)
    evp.evp_poisson_solve(sim.handle, rd, psi)
    sim.sync()
    ref = oracle.solve_poisson(r, g)
    got = psi.cpu().numpy().astype(np.float64)
    if not walls:
        got = got - got.mean()
        ref = ref - ref.mean()
    assert rel(got, ref) < tol


@pytest.mark.parametrize("shape", SHAPES)
def test_project_divergence_and_parity(evp, shape):
    sim, st, g, prm = setup_case(evp, shape, 'oldroyd_b', {}, evp.EVP_FP64)
    rng = np.random.default_rng(4)
    U, V, W = (rng.standard_normal(sim.shape) for _ in range(3))
    if shape[3]:
        V[:, -1] = 0.0
    sim.set_state(U, V, W)
    sim.project()
    code, bits, maxdiv = sim.sync()
    U2, V2, W2, _ = oracle.project(U, V, W, g, 1.0)
    for f, ref in ((evp.EVP_U, U2), (evp.EVP_V, V2), (evp.EVP_W, W2)):
        assert rel(sim.get(f), ref) < 1e-12
    assert maxdiv <= 1e-12 * max(1.0, np.abs(U).max() / g.dx)
    d = oracle.divergence(sim.get(evp.EVP_U), sim.get(evp.EVP_V), sim.get(evp.EVP_W), g)
    assert np.abs(d).max() <= 1e-12 * max(1.0, np.abs(U).max() / g.dx)


def fields(sim, evp):
    return ([sim.get(f) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P)]
            + [sim.get(evp.EVP_BXX + c) for c in range(6)])


def oracle_fields(st):
    return [st.U, st.V, st.W, st.p] + list(st.B)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("model,extra", MODELS)
def test_rk3_step_fp64(evp, shape, model, extra):
    # channel shapes carry the uniform body force of the Poiseuille problem
    dpdx = 0.05 if shape[3] else 0.0
    force = (dpdx, 0.0, 0.0) if dpdx else None
    sim, st, g, prm = setup_case(evp, shape, model, extra, evp.EVP_FP64, dpdx=dpdx)
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm, force)
    code, bits, maxdiv = sim.sync()
    for got, ref in zip(fields(sim, evp), oracle_fields(st)):
        assert rel(got, ref) < 1e-10
    assert maxdiv < 1e-11


@pytest.mark.parametrize("shape", SHAPES[:2])
@pytest.mark.parametrize("model,extra", MODELS)
def test_rk3_step_fp32(evp, shape, model, extra):
    """FP32 velocity and stress within 1e-5 of the FP64 oracle after one step.
    The pressure is recovered from div(u*)/(2 alpha dt): FP32 rounding of u*
    (relative eps32) leaves a spurious divergence ~ eps32 |u|/h, so psi carries an
    absolute error ~ eps32 |u| h / (2 alpha dt); it is checked against 8x that bound."""
    sim, st0, g, prm = setup_case(evp, shape, model, extra, evp.EVP_FP32)
    dt = 2e-3
    sim.step(dt)
    st = oracle.rk3_step(st0, dt, g, prm)
    sim.sync()
    got = fields(sim, evp)
    ref = oracle_fields(st)
    for q, (a, b) in enumerate(zip(got, ref)):
        if q == 3:
            continue
        assert rel(a, b) < 1e-5, (q, rel(a, b))
    eps32 = float(np.finfo(np.float32).eps)
    umax = max(np.abs(st0.U).max(), np.abs(st0.V).max(), np.abs(st0.W).max())
    h = max(g.dx, g.dy, g.dz)
    bound = 8.0 * sum(eps32 * umax * h / (2.0 * a * dt) for a in oracle.RK3_ALPHA)
    assert np.abs(got[3] - ref[3]).max() < bound


# rows of 128 cells or more (several 32-wide tiles per row, 144 = 4.5 tiles)
ROW_SHAPES = [(128, 12, 12, True), (128, 16, 8, False), (144, 10, 8, True)]


@pytest.mark.parametrize("shape", ROW_SHAPES)
@pytest.mark.parametrize("model,extra", [MODELS[2], MODELS[1]])
def test_rk3_step_long_rows_fp64(evp, shape, model, extra):
    """Two RK3 steps on long rows (walls: both wall rows and their ghost rules;
    periodic: the seams) within 1e-10 of the oracle."""
    dpdx = 0.05 if shape[3] else 0.0
    force = (dpdx, 0.0, 0.0) if dpdx else None
    sim, st, g, prm = setup_case(evp, shape, model, extra, evp.EVP_FP64, dpdx=dpdx)
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm, force)
    sim.sync()
    for got, ref in zip(fields(sim, evp), oracle_fields(st)):
        assert rel(got, ref) < 1e-10


@pytest.mark.parametrize("shape", ROW_SHAPES)
def test_rk3_step_long_rows_fp32(evp, shape):
    sim, st0, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, evp.EVP_FP32)
    dt = 2e-3
    sim.step(dt)
    st = oracle.rk3_step(st0, dt, g, prm)
    sim.sync()
    for q, (a, b) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if q != 3:
            assert rel(a, b) < 1e-5, (q, rel(a, b))


def test_c1_ten_steps_fp64(evp):
    """Single-phase Oldroyd-B Taylor-Green box, 32^3, Re = 1, Wi = 1, beta = 0.5,
    10 RK3 steps of dt = 1e-3: every field within 1e-10 of the oracle."""
    n, L = 32, 2 * np.pi
    geo = inputs.geometry(n, n, n, L, L, L)
    U, V, W = inputs.taylor_green(geo)
    sim = evp.Simulation(evp.make_grid(n, n, n, L, L, L), 'oldroyd_b',
                         evp.make_params(Re=1.0, Wi=1.0, beta=0.5, precision=evp.EVP_FP64))
    sim.set_state(U, V, W)
    g = oracle.Grid(n, n, n, L, L, L)
    st = oracle.State.rest(g, U, V, W)
    prm = oracle.Params.from_groups('oldroyd_b', 1.0, 1.0, 0.5)
    for _ in range(10):
        sim.step(1e-3)
        st = oracle.rk3_step(st, 1e-3, g, prm)
    code, bits, maxdiv = sim.sync()
    assert code == 0 and bits == 0
    for got, ref in zip(fields(sim, evp), oracle_fields(st)):
        assert rel(got, ref) < 1e-10
    assert maxdiv <= 1e-12


def test_nonfinite_input_raises_status(evp):
    n = 16
    sim = evp.Simulation(evp.make_grid(n, n, n, 1.0, 1.0, 1.0), 'oldroyd_b',
                         evp.make_params(Re=1.0, Wi=1.0, beta=0.5))
    U = np.zeros((n, n, n))
    U[3, 4, 5] = np.nan
    sim.set(evp.EVP_U, U)
    sim.step(1e-3)
    code, bits, _ = sim.sync(raise_on_error=False)
    assert code == evp.EVP_ERR_NONFINITE and bits & evp.EVP_BIT_NONFINITE
    # the state stays usable after the error is reported: once the velocity (which
    # the step filled with NaN, and whose divergence sync evaluates) is reset, the
    # next sync is clean
    for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W):
        sim.set(f, np.zeros((n, n, n)))
    code, bits, maxdiv = sim.sync(raise_on_error=False)
    assert code == 0 and bits == 0 and maxdiv == 0.0


@pytest.mark.parametrize("walls", [False, True])
def test_fp32_stress_front(evp, walls):
    """FP32 against the FP64 oracle across a sharp front of the conformation tensor:
    B_xx jumps by a factor of 100 (and B_xy by 5) over one cell on two x-planes and
    two z-planes, where the WENO5 smoothness indicators are large and the weights
    switch stencils.  Two RK3 steps, Oldroyd-B and Saramito."""
    shape = (32, 16, 16, walls)
    for model, extra in (('oldroyd_b', {}), ('saramito', {'Bi': 0.4})):
        sim, st, g, prm = setup_case(evp, shape, model, extra, evp.EVP_FP32)
        B = [b.copy() for b in st.B]
        front = np.zeros(sim.shape, dtype=bool)
        front[:, :, 8:20] = True
        front[4:9] = True
        B[0] = np.where(front, 100.0 * B[0], B[0])
        B[1] = np.where(front, 5.0 + B[1], B[1])           # B stays positive definite
        B = [b.astype(np.float32).astype(np.float64) for b in B]
        for c in range(6):
            sim.set(evp.EVP_BXX + c, B[c])
        st.B = B
        dt = 1e-3
        for _ in range(2):
            sim.step(dt)
            st = oracle.rk3_step(st, dt, g, prm)
        code, bits, _ = sim.sync(raise_on_error=False)
        assert bits & evp.EVP_BIT_NONFINITE == 0
        for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
            if q == 3:
                continue    # FP32 pressure: see test_rk3_step_fp32
            assert rel(got, ref) < 1e-5, (model, q, rel(got, ref))


@pytest.mark.parametrize("prec", [0, 1])
def test_three_substeps_equal_one_step(evp, prec):
    """evp_substep k = 0, 1, 2 runs the kernels of evp_step in the same order (the
    substep API also writes the last history, which the step skips): the fields
    agree bit for bit, including the summed stress handed from the stress kernel
    to the momentum kernel."""
    shape = (48, 24, 18, True)
    a_sim, _, _, _ = setup_case(evp, shape, 'fene_p', {'L2': 60.0}, prec)
    b_sim, _, _, _ = setup_case(evp, shape, 'fene_p', {'L2': 60.0}, prec)
    dt = 2e-3
    for _ in range(2):
        a_sim.step(dt)
        for k in range(3):
            evp.evp_substep(b_sim.handle, dt, k)
    a_sim.sync()
    b_sim.sync()
    for q, (x, y) in enumerate(zip(fields(a_sim, evp), fields(b_sim, evp))):
        assert np.array_equal(x, y), q


def test_batched_field_copies(evp):
    """evp_set_fields / evp_get_fields move the same data as the single-field
    calls (host and device buffers), apply the wall rule to v, and reject the
    read-only field before copying anything."""
    import torch
    shape = (32, 16, 8, True)
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, evp.EVP_FP32)
    rng = np.random.default_rng(21)
    fields = [evp.EVP_U, evp.EVP_V, evp.EVP_P, evp.EVP_BXY]
    vals = [rng.standard_normal(sim.shape).astype(np.float32) for _ in fields]
    evp.evp_set_fields(sim.handle, fields, vals)
    out = [np.empty(sim.shape, np.float32) for _ in fields]
    evp.evp_get_fields(sim.handle, fields, out)
    for f, v, o in zip(fields, vals, out):
        ref = v.copy()
        if f == evp.EVP_V:
            ref[:, -1] = 0.0        # the stored top face is the wall
        assert np.array_equal(o, ref), f
        single = np.empty(sim.shape, np.float32)
        evp.evp_get_field(sim.handle, f, single)
        assert np.array_equal(single, o)
    dev = [torch.zeros(sim.shape, dtype=torch.float32, device='cuda') for _ in fields]
    evp.evp_get_fields(sim.handle, fields, dev)
    for d, o in zip(dev, out):
        assert np.array_equal(d.cpu().numpy(), o)
    with pytest.raises(evp.EvpError):
        evp.evp_set_fields(sim.handle, [evp.EVP_U, evp.EVP_PSI], [vals[0], vals[0]])
    got = np.empty(sim.shape, np.float32)
    evp.evp_get_field(sim.handle, evp.EVP_U, got)
    assert np.array_equal(got, out[0])          # nothing copied by the rejected call
    evp.evp_set_fields(sim.handle, [], [])      # an empty batch is a no-op


def test_bad_arguments_rejected(evp):
    with pytest.raises(evp.EvpError):
        evp.Simulation(evp.make_grid(20, 16, 16, 1.0, 1.0, 1.0), 'oldroyd_b', evp.make_params(Re=1.0))
    with pytest.raises(evp.EvpError):
        evp.Simulation(evp.make_grid(16, 16, 16, 1.0, 1.0, 1.0), 'fene_p', evp.make_params(Re=1.0, L2=2.0))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_volume_penalisation_channel(evp, prec, tol):
    """Volume-penalisation IBM (Sec. 3.3.2, Eq. forceAdded): a driven Oldroyd-B
    channel around a fixed solid block; three RK3 steps against the oracle."""
    nx, ny, nz = 48, 24, 16
    geo = inputs.geometry(nx, ny, nz, 4.0, 2.0, 2.0, True)
    g = oracle.Grid(nx, ny, nz, 4.0, 2.0, 2.0, True)
    block = lambda x, y, z: ((np.abs(x - 2.0) < 0.5) & (np.abs(y + 0.2) < 0.4) & (np.abs(z - 1.0) < 0.6)).astype(float)
    al = inputs.solid_fractions(geo, block)
    U, V, W = inputs.poiseuille(geo)
    B = inputs.random_conformation(geo, 8, amp=0.2)
    prm = oracle.Params.from_groups('oldroyd_b', 10.0, 0.5, 0.5)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, 4.0, 2.0, 2.0, True), 'oldroyd_b',
                         evp.make_params(Re=10.0, Wi=0.5, beta=0.5, dpdx=0.2, precision=prec, penalization=1))
    sim.set_state(U, V, W, B=B)
    for q, f in enumerate((evp.EVP_SOLID_X, evp.EVP_SOLID_Y, evp.EVP_SOLID_Z)):
        sim.set(f, al[q])
    rd = (lambda a: a.astype(np.float32).astype(np.float64)) if prec else (lambda a: a)
    st = oracle.State.rest(g, rd(U), rd(V), rd(W))
    st.B = [rd(b) for b in B]
    solid = tuple(rd(a) for a in al)
    for _ in range(3):
        sim.step(5e-3)
        st = oracle.rk3_step(st, 5e-3, g, prm, (0.2, 0.0, 0.0), solid)
    sim.sync()
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec and q == 3:
            continue   # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < tol, (q, rel(got, ref))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_abc_forcing_fene_p(evp, prec, tol):
    """ABC body force A(sin kz + cos ky, sin kx + cos kz, sin ky + cos kx) on a
    FENE-P box (the forced-turbulence setting): two RK3 steps against the oracle,
    the force sampled at the faces from its definition.  In FP32 (nx a multiple of
    4) the momentum kernel computes two cells per thread and reads the force tables
    in pairs."""
    nx, ny, nz = 48, 24, 18
    L = 2 * np.pi
    geo = inputs.geometry(nx, ny, nz, L, L, L)
    g = oracle.Grid(nx, ny, nz, L, L, L)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, 21, 3), 1.0)
    if prec == 1:
        U, V, W = (a.astype(np.float32).astype(np.float64) for a in (U, V, W))
    A, k = 0.7, 2.0
    xc, yc, zc = g.xc(), g.yc(), g.zc()
    force = (A * (np.sin(k * zc) + np.cos(k * yc)) + 0 * g.zeros(), A * (np.sin(k * xc) + np.cos(k * zc)) + 0 * g.zeros(),
             A * (np.sin(k * yc) + np.cos(k * xc)) + 0 * g.zeros())
    prm = oracle.Params.from_groups('fene_p', 200.0, 5.0, 0.9, L2=900.0)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, L, L, L), 'fene_p',
                         evp.make_params(Re=200.0, Wi=5.0, beta=0.9, L2=900.0, abc_amp=A, abc_k=k, precision=prec))
    sim.set_state(U, V, W)
    st = oracle.State.rest(g, U, V, W)
    for _ in range(2):
        sim.step(1e-3)
        st = oracle.rk3_step(st, 1e-3, g, prm, force)
    sim.sync()
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec == 1 and q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < tol, (q, rel(got, ref))


def defect_conformation(geo, seed, L2):
    """B near I, with one ball where tr B is about 0.97 L^2 (the FENE-P trace trigger)
    and one ball where B_xx < 0 (det B < 0); every cell is far from both thresholds."""
    B = inputs.random_conformation(geo, seed, amp=0.3)
    y0 = -geo['ly'] / 2 if geo['walls_y'] else 0.0
    cy = y0 + 0.5 * geo['ly']
    ball_a = inputs.sphere_distance(geo, (0.3 * geo['lx'], cy, 0.3 * geo['lz']), 0.22 * geo['lz']) < 0
    ball_b = inputs.sphere_distance(geo, (0.7 * geo['lx'], cy, 0.7 * geo['lz']), 0.22 * geo['lz']) < 0
    for c in (0, 3, 5):
        B[c] = np.where(ball_a, B[c] + (0.97 * L2 - 3.0) / 3.0, B[c])
    B[0] = np.where(ball_b, B[0] - 2.0, B[0])
    return B, ball_a, ball_b


def diffusion_case(evp, shape, precision, art):
    nx, ny, nz, walls = shape
    L2 = 60.0
    sim, st, g, prm = setup_case(evp, shape, 'fene_p', {'L2': L2, 'art_diff': art}, precision)
    geo = inputs.geometry(nx, ny, nz, g.lx, g.ly, g.lz, walls)
    B, ball_a, ball_b = defect_conformation(geo, 11, L2)
    if precision == evp.EVP_FP32:
        B = [b.astype(np.float32).astype(np.float64) for b in B]
    sim.set_state(B=B)
    st.B = [b.copy() for b in B]
    # both sides select the same cells: no cell within reach of a threshold
    det = oracle.determinant(B)
    tr = B[0] + B[3] + B[5]
    assert ball_a.any() and ball_b.any() and (det < 0).sum() == ball_b.sum()
    assert np.abs(det).min() > 1e-2 and np.abs(tr - 0.95 * L2).min() > 0.1
    return sim, st, g, prm


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1]])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_artificial_diffusion_rhs(evp, shape, prec, tol):
    """Sec. 3.1 local artificial diffusion in the stress right-hand side: FENE-P
    with cells over 0.95 L^2 and cells with det B < 0."""
    import torch
    sim, st, g, prm = diffusion_case(evp, shape, prec, 0.05)
    out = torch.empty((6,) + sim.shape, dtype=torch.float32 if prec else torch.float64, device='cuda')
    evp.evp_stress_rhs(sim.handle, out)
    sim.sync()
    ref = oracle.stress_rhs(st.U, st.V, st.W, st.B, g, prm)
    plain = oracle.stress_rhs(st.U, st.V, st.W, st.B, g, oracle.Params.from_groups('fene_p', 2.0, 0.8, 0.4, L2=60.0))
    assert max(np.abs(r - q).max() for r, q in zip(ref, plain)) > 1e-2   # the term is present
    for c in range(6):
        assert rel(out[c].cpu().numpy(), ref[c]) < tol, (c, rel(out[c].cpu().numpy(), ref[c]))


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1]])
def test_artificial_diffusion_steps_fp64(evp, shape):
    sim, st, g, prm = diffusion_case(evp, shape, evp.EVP_FP64, 0.02)
    dt = 1e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm)
    code, bits, _ = sim.sync()
    assert code == evp.EVP_OK and bits & evp.EVP_BIT_DET_NEG     # reported, not an error
    for f, ref in [(evp.EVP_U, st.U), (evp.EVP_V, st.V), (evp.EVP_W, st.W), (evp.EVP_P, st.p)] + \
            [(evp.EVP_BXX + c, st.B[c]) for c in range(6)]:
        assert rel(sim.get(f), ref) < 1e-10, (f, rel(sim.get(f), ref))


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1]])
def test_fp32_residual_is_the_fp64_divergence_of_the_stored_fields(evp, shape):
    """The residual evp_sync reports after an FP32 step is max |div u| of the FP32
    velocity the step stored, evaluated in FP64 (to the rounding of that sum)."""
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, evp.EVP_FP32)
    for _ in range(2):
        sim.step(2e-3)
    code, bits, maxdiv = sim.sync()
    U, V, W = (sim.get(f).astype(np.float64) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W))
    host = np.abs(oracle.divergence(U, V, W, g)).max()
    # the terms are ~|u|/h while their sum is at the FP32 rounding level: allow a
    # few FP64 ulps of the terms (an FP32-rounded evaluation would be ~1e8 times off)
    terms = np.abs(U).max() / g.dx + np.abs(V).max() / g.dy + np.abs(W).max() / g.dz
    assert host > 0 and abs(maxdiv - host) <= 8 * 2.0 ** -52 * terms, (maxdiv, host, terms)


def test_device_conversion_selftest(evp):
    """The integer-operation FP32 <-> FP64 conversions of the FP64 residual and the
    FP32 Thomas sweep agree with the conversion instructions (bit for bit outside
    the binary32 subnormal range)."""
    assert evp.evp_selftest() == 0


@pytest.mark.parametrize("shape", [(18, 12, 16, True), (54, 12, 8, False)])
@pytest.mark.parametrize("prec", [0, 1])
def test_rk3_step_rows_not_16_byte_multiples(evp, shape, prec):
    """nx = 18 or 54: FP32 rows are not a whole number of 16-byte chunks, so the
    kernels stage their tiles element by element; the step still matches the oracle."""
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, prec)
    dt = 2e-3
    sim.step(dt)
    st = oracle.rk3_step(st, dt, g, prm)
    sim.sync()
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec == 1 and q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < (1e-10 if prec == 0 else 1e-5), (q, rel(got, ref))


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("shape,model,extra,prec", [(SHAPES[1], 'saramito', {'Bi': 0.4}, 1),
                                                    (SHAPES[0], 'fene_p', {'L2': 60.0}, 0)])
def test_programmatic_dependent_launch_changes_nothing(evp, graph, shape, model, extra, prec):
    """Two RK3 steps with programmatic dependent launch on and off, launched directly
    or replayed as a CUDA graph, give bit-identical fields."""
    out = []
    for pdl in (True, False):
        sim, st, g, prm = setup_case(evp, shape, model, extra, prec)
        evp.evp_set_pdl(sim.handle, pdl)
        evp.evp_set_graph(sim.handle, graph)
        for _ in range(2):
            sim.step(2e-3)
        sim.sync()
        out.append(fields(sim, evp))
        sim.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("graph", [False, True])
def test_nvtx_ranges_change_nothing(evp, graph):
    """NVTX ranges on (steps, substeps, kernels) with and without kernel timing give
    the fields of a run without them, bit for bit, and the kernel timing still
    counts every launch."""
    out = []
    for nvtx, timing in ((False, False), (True, False), (True, True)):
        sim, st, g, prm = setup_case(evp, SHAPES[1], 'saramito', {'Bi': 0.4}, evp.EVP_FP32)
        evp.evp_set_nvtx(sim.handle, nvtx)
        evp.evp_set_graph(sim.handle, graph)
        if timing:
            evp.evp_kernel_timing(sim.handle, True)
        for _ in range(2):
            sim.step(2e-3)
        sim.substep(2e-3, 0)
        sim.sync()
        if timing:
            times = evp.evp_kernel_times(sim.handle)
            assert times['stress_weno_update'][1] == 7 and times['project_correct'][1] == 7
        out.append(fields(sim, evp))
        sim.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            np.testing.assert_array_equal(a, b)


def implicit_case(evp, shape, prec, model='oldroyd_b', extra=None):
    extra = extra or {}
    nx, ny, nz, walls = shape
    sim0, st, g, prm = setup_case(evp, shape, model, extra, prec)
    sim0.close()
    ly = 2.0 if walls else 2 * np.pi
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls), model,
                         evp.make_params(Re=2.0, Wi=0.8, beta=0.4, precision=prec, viscous_implicit=1, **extra))
    sim.set_state(st.U, st.V, st.W, st.p, st.B)
    return sim, st, g, prm


@pytest.mark.parametrize("shape", SHAPES)
def test_implicit_viscous_steps_fp64(evp, shape):
    """Eq. NS-num1 read literally (Helmholtz solve per component and substep):
    two RK3 steps against the oracle, FP64."""
    sim, st, g, prm = implicit_case(evp, shape, evp.EVP_FP64, 'saramito', {'Bi': 0.4})
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm, implicit_viscous=True)
    code, bits, maxdiv = sim.sync()
    for got, ref in zip(fields(sim, evp), oracle_fields(st)):
        assert rel(got, ref) < 1e-10, rel(got, ref)
    assert maxdiv < 1e-11


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_implicit_viscous_step_fp32(evp, shape):
    sim, st, g, prm = implicit_case(evp, shape, evp.EVP_FP32)
    dt = 2e-3
    sim.step(dt)
    st = oracle.rk3_step(st, dt, g, prm, implicit_viscous=True)
    sim.sync()
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < 1e-5, (q, rel(got, ref))


def test_implicit_viscous_channel_mode_decay(evp):
    """A no-slip shear mode u_j = sin(pi m (j + 1/2)/ny) decays by the closed-form
    Crank-Nicolson factor prod_k (1 - a_k dt nu lam)/(1 + a_k dt nu lam) per step,
    here over 5 steps with a dt 20 times the explicit viscous limit."""
    nx, ny, nz = 8, 24, 8
    m, Re = 2, 10.0
    nu, dy = 1.0 / Re, 2.0 / ny
    U = np.broadcast_to(np.sin(np.pi * m * (np.arange(ny) + 0.5) / ny)[None, :, None], (nz, ny, nx)).copy()
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, 1.0, 2.0, 1.0, True), 'newtonian',
                         evp.make_params(Re=Re, beta=1.0, viscous_implicit=1))
    sim.set_state(U=U)
    lam = (2 - 2 * np.cos(np.pi * m / ny)) / dy ** 2
    dt = 20 * dy ** 2 / (6 * nu)
    f = 1.0
    for a in oracle.RK3_ALPHA:
        f *= (1 - a * dt * nu * lam) / (1 + a * dt * nu * lam)
    for _ in range(5):
        sim.step(dt)
    sim.sync()
    np.testing.assert_allclose(sim.get(evp.EVP_U), U * f ** 5, rtol=0, atol=1e-12)


PARTICLES = [((0.72, 0.95, 1.1), 0.3, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
             ((1.35, 1.05, 0.55), 0.25, (0.2, -0.1, 0.05), (0.3, -0.4, 1.5))]


def particle_case(evp, prec, walls=False):
    n = 32
    shape = (n, 24, 16, True) if walls else (n, n, n, False)
    nx, ny, nz, _ = shape
    lx, ly, lz = (2.0, 1.5, 1.0) if walls else (2.0, 2.0, 2.0)
    geo = inputs.geometry(nx, ny, nz, lx, ly, lz, walls)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, 5, 3), 1.0)
    if walls:
        U = U + inputs.poiseuille(geo)[0]
    g = oracle.Grid(nx, ny, nz, lx, ly, lz, walls)
    prm = oracle.Params.from_groups('oldroyd_b', Re=5.0, Wi=0.8, beta=0.4)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, lx, ly, lz, walls), 'oldroyd_b',
                         evp.make_params(Re=5.0, Wi=0.8, beta=0.4, precision=prec))
    parts = PARTICLES if not walls else [((1.0, 0.05, 0.5), 0.3, (0.1, 0.0, 0.0), (0.0, 0.0, 0.8))]
    sim.set_state(U, V, W)
    evp.evp_set_particles(sim.handle, parts, iters=3)
    st = oracle.State.rest(g, U, V, W)
    if prec == evp.EVP_FP32:
        rd = lambda a: a.astype(np.float32).astype(np.float64)
        st.U, st.V, st.W = rd(st.U), rd(st.V), rd(st.W)
    if walls:
        st.V[:, -1] = 0.0
    st.particles = [{'centre': c, 'radius': r, 'u': u, 'omega': w} for c, r, u, w in parts]
    return sim, st, g, prm, len(parts)


@pytest.mark.parametrize("walls", [False, True])
def test_ibm_particles_fp64(evp, walls):
    """Discrete-forcing IBM (Eqs. IBM a-d, CoVe2) with a fixed and a moving,
    spinning sphere: two RK3 steps against the oracle, fields, centres, forces."""
    sim, st, g, prm, n = particle_case(evp, evp.EVP_FP64, walls)
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm)
    code, bits, maxdiv = sim.sync()
    for got, ref in zip(fields(sim, evp), oracle_fields(st)):
        assert rel(got, ref) < 1e-10, rel(got, ref)
    assert maxdiv < 1e-11
    out = evp.evp_get_particles(sim.handle, n)
    for p in range(n):
        np.testing.assert_allclose(out[p, :3], st.particles[p]['centre'], rtol=0, atol=1e-14)
        ft = np.concatenate(st.particle_forces[p])
        assert np.abs(out[p, 9:] - ft).max() < 1e-9 * np.abs(ft).max(), (out[p, 9:], ft)


def test_ibm_particles_fp32(evp):
    sim, st, g, prm, n = particle_case(evp, evp.EVP_FP32)
    dt = 2e-3
    sim.step(dt)
    st = oracle.rk3_step(st, dt, g, prm)
    sim.sync()
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < 1e-5, (q, rel(got, ref))


def test_ibm_rejects_bad_particles(evp):
    sim = evp.Simulation(evp.make_grid(32, 24, 16, 2.0, 1.5, 1.0, True), 'newtonian', evp.make_params(Re=5.0))
    for bad in ([((1.0, 0.0, 0.5), 0.1, (0, 0, 0), (0, 0, 0))],          # radius below 2 dx
                [((1.0, 0.5, 0.5), 0.3, (0, 0, 0), (0, 0, 0))]):          # too close to the top wall
        with pytest.raises(evp.EvpError) as e:
            evp.evp_set_particles(sim.handle, bad)
        assert e.value.code == evp.EVP_ERR_ARG
    sim2 = evp.Simulation(evp.make_grid(32, 24, 16, 2.0, 2.0, 1.0, True), 'newtonian', evp.make_params(Re=5.0))
    with pytest.raises(evp.EvpError):
        evp.evp_set_particles(sim2.handle, [((1.0, 0.0, 0.5), 0.3, (0, 0, 0), (0, 0, 0))])   # non-cubic cells
    evp.evp_set_particles(sim.handle, [])


@pytest.mark.parametrize("prec", [0, 1])
def test_ibm_free_particles(evp, prec):
    """Free spheres (Newton-Euler with the inner-fluid integrals, gravity along -y):
    a heavy one released in a shear flow and a light spinning one; two RK3 steps
    against the oracle: fields, centres, velocities, angular velocities."""
    n, L = 32, 2.0
    geo = inputs.geometry(n, n, n, L, L, L)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, 9, 3), 0.5)
    g = oracle.Grid(n, n, n, L, L, L)
    prm = oracle.Params.from_groups('oldroyd_b', Re=5.0, Wi=0.8, beta=0.4)
    sim = evp.Simulation(evp.make_grid(n, n, n, L, L, L), 'oldroyd_b',
                         evp.make_params(Re=5.0, Wi=0.8, beta=0.4, precision=prec, gravity=3.0))
    parts = [((0.7, 1.1, 0.9), 0.3, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), 2.5),
             ((1.4, 0.8, 1.3), 0.25, (0.1, 0.0, -0.1), (0.0, 0.0, 2.0), 0.8)]
    sim.set_state(U, V, W)
    evp.evp_set_particles(sim.handle, parts, iters=3)
    st = oracle.State.rest(g, U, V, W)
    if prec == evp.EVP_FP32:
        rd = lambda a: a.astype(np.float32).astype(np.float64)
        st.U, st.V, st.W = rd(st.U), rd(st.V), rd(st.W)
    st.particles = [{'centre': c, 'radius': r, 'u': u, 'omega': w, 'rho': d} for c, r, u, w, d in parts]
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm, gravity=3.0)
    sim.sync()
    tol = 1e-10 if prec == 0 else 1e-5
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec == 1 and q == 3:
            continue
        assert rel(got, ref) < tol, (q, rel(got, ref))
    out = evp.evp_get_particles(sim.handle, 2)
    for p in range(2):
        ref = st.particles[p]
        assert np.abs(out[p, :3] - ref['centre']).max() < (1e-13 if prec == 0 else 1e-7)
        for a, b in ((out[p, 3:6], ref['u']), (out[p, 6:9], ref['omega'])):
            assert np.abs(a - np.asarray(b)).max() < (1e-9 if prec == 0 else 1e-4) * max(1.0, np.abs(b).max()), (a, b)



@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1]])
@pytest.mark.parametrize("prec", [0, 1])
def test_soft_particles(evp, shape, prec):
    """Soft particle (one continuum, neo-Hookean, Sec. 3.3.2): the solid fraction of
    a smoothed sphere is advected like B and the stress is phi_s G (B - I); two RK3
    steps against the oracle."""
    nx, ny, nz, walls = shape
    sim0, st, g, prm = setup_case(evp, shape, 'neo_hookean', {}, prec)
    sim0.close()
    ly = 2.0 if walls else 2 * np.pi
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
    cy = 0.0 if walls else np.pi
    d = inputs.sphere_distance(geo, (np.pi, cy, np.pi), 1.6 if not walls else 0.6)
    phis = np.clip(0.5 - d / (3.0 * g.dx), 0.0, 1.0)
    if prec == evp.EVP_FP32:
        phis = phis.astype(np.float32).astype(np.float64)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls), 'neo_hookean',
                         evp.make_params(Re=2.0, Wi=0.8, beta=0.4, precision=prec, soft_particles=1))
    sim.set_state(st.U, st.V, st.W, st.p, st.B)
    sim.set(evp.EVP_PHI, phis)
    st.phis, st.phis_hist = phis.copy(), np.zeros(g.shape)
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm)
    sim.sync()
    tol = 1e-10 if prec == 0 else 1e-5
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec == 1 and q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < tol, (q, rel(got, ref))
    assert rel(sim.get(evp.EVP_PHI), st.phis) < tol


ODD_SHAPES = [(24, 9, 27, False), (16, 7, 9, True)]


@pytest.mark.parametrize("shape", ODD_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_rk3_step_odd_sizes(evp, shape, prec):
    """Odd counts: a periodic ny = 9 and nz = 27 (radix-3 FFTs, an unpaired real
    line in the x transforms), and a wall-bounded ny = 7 with nz = 9."""
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, prec)
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm)
    sim.sync()
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec == 1 and q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        assert rel(got, ref) < (1e-10 if prec == 0 else 1e-5), (q, rel(got, ref))


@pytest.mark.parametrize("shape", ODD_SHAPES)
def test_poisson_solve_odd_sizes(evp, shape):
    import torch
    nx, ny, nz, walls = shape
    sim, st, g, prm = setup_case(evp, shape, 'oldroyd_b', {}, evp.EVP_FP64)
    r = np.random.default_rng(12).standard_normal((nz, ny, nx))
    r -= r.mean()
    rd = torch.tensor(r, dtype=torch.float64, device='cuda')
    psi = torch.empty_like(rd)
    evp.evp_poisson_solve(sim.handle, rd, psi)
    sim.sync()
    ref = oracle.solve_poisson(r, g)
    got = psi.cpu().numpy()
    if not walls:
        got, ref = got - got.mean(), ref - ref.mean()
    assert rel(got, ref) < 1e-12


# power-of-two sizes 16 .. 256 in each role (x pass, z pass, periodic y solve) of the
# register-resident FFT kernels, with walls and periodic
POW2_SHAPES = [(256, 16, 128, False), (16, 256, 64, False), (128, 64, 256, False), (64, 128, 16, False),
               (256, 24, 128, True), (128, 16, 256, True), (16, 8, 64, True)]


@pytest.mark.parametrize("shape", POW2_SHAPES)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_poisson_solve_power_of_two_sizes(evp, shape, prec, tol):
    import torch
    nx, ny, nz, walls = shape
    sim, st, g, prm = setup_case(evp, shape, 'oldroyd_b', {}, prec)
    r = np.random.default_rng(13).standard_normal((nz, ny, nx))
    r -= r.mean()
    if prec == 1:
        r = r.astype(np.float32).astype(np.float64)
    rd = torch.tensor(r, dtype=torch.float32 if prec else torch.float64, device='cuda')
    psi = torch.empty_like(rd)
    evp.evp_poisson_solve(sim.handle, rd, psi)
    sim.sync()
    ref = oracle.solve_poisson(r, g)
    got = psi.cpu().numpy().astype(np.float64)
    if not walls:
        got, ref = got - got.mean(), ref - ref.mean()
    assert rel(got, ref) < tol, (shape, prec, rel(got, ref))


@pytest.mark.parametrize("thomas_fp64", [0, 1])
@pytest.mark.parametrize("shape", [(16, 512, 8, True), (32, 128, 16, True), (8, 36, 8, True)])
def test_fp32_wall_solve_of_the_lowest_modes_is_rounding_exact(evp, shape, thomas_fp64):
    """The (kx, kz) = (0, 0) system of a wall-bounded solve is the pinned 1-D
    Neumann Laplacian, whose condition number grows like ny^2 (about 1e5 at 512
    rows): a plain FP32 sweep loses about five digits on it.  A right-hand side
    that varies in y only reaches the FP32 solve through exact x and z
    transforms, so the FP32 result must be the FP64 solution of the same
    (FP32-rounded) data rounded once: within 2 ulps of the oracle, and within 1
    ulp of the FP64 state's own solve; with the double-single sweep (default) and
    with the FP64 sweep (thomas_fp64 = 1)."""
    import torch
    nx, ny, nz, walls = shape
    rng = np.random.default_rng(21)
    prof = rng.standard_normal(ny) + np.cos(np.pi * (np.arange(ny) + 0.5) / ny)
    r = np.ascontiguousarray(np.broadcast_to(prof[None, :, None], (nz, ny, nx)), dtype=np.float32).astype(np.float64)
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, 2.0, 2 * np.pi, walls)
    g = oracle.Grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls)
    out = {}
    for prec in (evp.EVP_FP32, evp.EVP_FP64):
        sim = evp.Simulation(evp.make_grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls), 'oldroyd_b',
                             evp.make_params(Re=2.0, Wi=0.8, beta=0.4, precision=prec, thomas_fp64=thomas_fp64))
        rd = torch.tensor(r, dtype=torch.float32 if prec else torch.float64, device='cuda').contiguous()
        psi = torch.empty(rd.shape, dtype=rd.dtype, device='cuda')
        evp.evp_poisson_solve(sim.handle, rd, psi)
        sim.sync()
        out[prec] = psi.cpu().numpy().astype(np.float64)
        sim.close()
    ref = oracle.solve_poisson(r, g)
    scale = np.abs(ref).max()
    ulp = np.spacing(np.float32(scale)).astype(np.float64)
    assert np.abs(out[evp.EVP_FP32] - ref).max() <= 2 * ulp, np.abs(out[evp.EVP_FP32] - ref).max() / ulp
    assert np.abs(out[evp.EVP_FP32] - out[evp.EVP_FP64]).max() <= ulp


@pytest.mark.parametrize("implicit", [0, 1])
def test_fp32_thomas_sweeps_agree(evp, implicit):
    """An FP32 channel stepped with the double-single and with the FP64 Thomas
    sweep (with the implicit viscous option: the Helmholtz tables too): the two
    runs' fields agree to FP32 rounding after three steps."""
    out = []
    for t in (0, 1):
        nx, ny, nz, walls = SHAPES[1]
        sim, st, g, prm = setup_case(evp, SHAPES[1], 'saramito', {'Bi': 0.4}, evp.EVP_FP32)
        sim.close()
        geo = inputs.geometry(nx, ny, nz, 2 * np.pi, 2.0, 2 * np.pi, walls)
        sim = evp.Simulation(evp.make_grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls), 'saramito',
                             evp.make_params(Re=2.0, Wi=0.8, beta=0.4, Bi=0.4, precision=evp.EVP_FP32,
                                             thomas_fp64=t, viscous_implicit=implicit))
        sim.set_state(st.U, st.V, st.W, st.p, st.B)
        for _ in range(3):
            sim.step(2e-3)
        sim.sync()
        out.append(fields(sim, evp))
        sim.close()
    for q, (a, b) in enumerate(zip(*out)):
        # the pressure accumulates psi, which carries the FP32 rounding of u*/dt
        tol = 1e-5 if q == 3 else 1e-6
        assert rel(a, b.astype(np.float64)) < tol, (q, rel(a, b.astype(np.float64)))


def test_fene_p_trace_limit_is_reported(evp):
    """A FENE-P state stretched beyond L^2 raises EVP_BIT_TRACE_LIMIT and evp_sync
    returns EVP_ERR_UNPHYSICAL (no clamping, no fault)."""
    n, L2 = 16, 30.0
    sim = evp.Simulation(evp.make_grid(n, n, n, 1.0, 1.0, 1.0), 'fene_p', evp.make_params(Re=1.0, L2=L2))
    big = np.full((n, n, n), 1.02 * L2 / 3.0)
    zero = np.zeros((n, n, n))
    sim.set_state(B=[big, zero, zero, big, zero, big])
    sim.step(1e-4)
    code, bits, _ = sim.sync(raise_on_error=False)
    assert code == evp.EVP_ERR_UNPHYSICAL and bits & evp.EVP_BIT_TRACE_LIMIT


# the longest transform in each role (512: x pass, periodic y solve, z pass, and a
# wall-normal y of 512 for the Thomas solve), with the other axes at their minimum,
# and the smallest grid the library accepts (nx = nz = 8, ny = 4 between walls)
EXTREME_SHAPES = [(512, 8, 8, False), (8, 512, 8, False), (8, 8, 512, False), (16, 512, 8, True), (8, 4, 8, True)]


@pytest.mark.parametrize("shape", EXTREME_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_poisson_solve_extreme_lengths(evp, shape, prec):
    """FP64 1e-12; FP32 2e-6 for transforms of up to 256 points (8 radix-2 stages,
    as above) scaled by the stage count log2(n) / 8, the growth of the FFT's rounding
    error with its length."""
    import torch
    nx, ny, nz, walls = shape
    sim, st, g, prm = setup_case(evp, shape, 'oldroyd_b', {}, prec)
    r = np.random.default_rng(14).standard_normal((nz, ny, nx))
    r -= r.mean()
    if prec == 1:
        r = r.astype(np.float32).astype(np.float64)
    rd = torch.tensor(r, dtype=torch.float32 if prec else torch.float64, device='cuda')
    psi = torch.empty_like(rd)
    evp.evp_poisson_solve(sim.handle, rd, psi)
    sim.sync()
    ref = oracle.solve_poisson(r, g)
    got = psi.cpu().numpy().astype(np.float64)
    if not walls:
        got, ref = got - got.mean(), ref - ref.mean()
    tol = 1e-12 if prec == 0 else 2e-6 * max(1.0, np.log2(max(nx, nz, 8 if walls else ny)) / 8.0)
    print('poisson', shape, prec, rel(got, ref))
    assert rel(got, ref) < tol, (shape, prec, rel(got, ref))


@pytest.mark.parametrize("shape", EXTREME_SHAPES)
@pytest.mark.parametrize("prec", [0, 1])
def test_rk3_step_extreme_lengths(evp, shape, prec):
    """One Saramito RK3 step on the extreme grids: FP64 1e-10, FP32 1e-5.  The
    viscous term is explicit (Reading 3), and RK3 is stable for it while
    dt 4 mu_s (1/dx^2 + 1/dy^2 + 1/dz^2) <= 2.51; dt is a quarter of that limit here
    (at most 2e-3).  Beyond it a step amplifies rounding in the shortest modes, by
    about 1e4 at 512 rows between walls with dt = 2e-3 (FP32 1e-3, FP64 8e-13
    relative), which would measure the scheme's instability, not the kernels."""
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, prec)
    lap = 4.0 * prm.mu_s * (1.0 / g.dx ** 2 + 1.0 / g.dy ** 2 + 1.0 / g.dz ** 2)
    dt = min(2e-3, 0.25 * 2.51 / lap)
    sim.step(dt)
    st = oracle.rk3_step(st, dt, g, prm)
    sim.sync()
    worst = 0.0
    for q, (got, ref) in enumerate(zip(fields(sim, evp), oracle_fields(st))):
        if prec == 1 and q == 3:
            continue    # FP32 pressure: see test_rk3_step_fp32
        worst = max(worst, rel(got, ref))
        assert rel(got, ref) < (1e-10 if prec == 0 else 1e-5), (q, rel(got, ref))
    print('rk3 step', shape, prec, worst)


@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[1]])
def test_checkpoint_and_resume_bitwise_fp64(evp, shape):
    """Checkpoint / resume of an RK3 state through the field copies: every field a
    state holds (velocity, pressure, conformation, both histories) read after two
    steps and written into a fresh state; both then take three more steps and agree
    bit for bit."""
    sim, st, g, prm = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, evp.EVP_FP64, dpdx=0.05 if shape[3] else 0.0)
    for _ in range(2):
        sim.step(2e-3)
    ids = [evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P] + [evp.EVP_BXX + c for c in range(6)]
    ids += [evp.EVP_RT_XX + c for c in range(6)] + [evp.EVP_NH_X + c for c in range(3)]
    saved = [sim.get(f) for f in ids]
    twin = evp.Simulation(sim.grid, 'saramito', sim.params)
    for f, a in zip(ids, saved):
        twin.set(f, a)
    for _ in range(3):
        sim.step(2e-3)
        twin.step(2e-3)
    for f in ids:
        assert np.array_equal(sim.get(f), twin.get(f)), f
    twin.close()
    sim.close()


def test_step_io_equals_copies_and_step(evp):
    """evp_step_io (copies in, one step, copies out, nothing waited for) gives what
    evp_set_fields + evp_step + evp_get_fields give, bit for bit, with two states on
    two streams stepping in turn and sharing nothing."""
    import torch
    shape = SHAPES[1]
    ids = [evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P] + [evp.EVP_BXX + c for c in range(6)]
    ref, _, _, _ = setup_case(evp, shape, 'saramito', {'Bi': 0.4}, evp.EVP_FP32, dpdx=0.05)
    start = [ref.get(f) for f in ids]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sims, ios, bufs = [], [], []
    for st in streams:
        sim = evp.Simulation(ref.grid, 'saramito', ref.params, stream=st.cuda_stream)
        b = [torch.from_numpy(a.copy()).pin_memory() for a in start]
        outs = [torch.empty_like(x).pin_memory() for x in b]
        ios.append(evp.StepIO(ids, [x.numpy() for x in b], ids, [x.numpy() for x in outs]))
        sims.append(sim)
        bufs.append((b, outs))
    for k in range(6):
        evp.evp_step_io(sims[k & 1].handle, 2e-3, ios[k & 1])
    torch.cuda.synchronize()
    for sim, (b, outs) in zip(sims, bufs):
        # each state restarted from `start` every step: its outputs are one step from it
        one = [sim.get(f) for f in ids]
        for a, o in zip(one, outs):
            assert np.array_equal(a, o.numpy())
    ref.set_state(*start[:4], B=start[4:])
    ref.step(2e-3)
    for f, o in zip(ids, bufs[0][1]):
        assert np.array_equal(ref.get(f), o.numpy()), f
    for s in sims + [ref]:
        s.close()
