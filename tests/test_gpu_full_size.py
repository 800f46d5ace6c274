"""Parity at the full sizes of the benchmark workloads, in the launch configuration
that the benchmark times: FP32 storage and the kernels of one RK3 substep exactly as
the step graph captures them (the graph replays these substep launches; graph and
direct launches are compared bit for bit in test_gpu_parity).

The oracle takes about half a minute per substep at 256x128x128, so the local parts
of the substep are checked on sampled outputs (windows, see oracle_windows; the
method is pinned by test_oracle_windows):
  * B^k (Eq. rk3tau) at every cell of each window's interior;
  * u* (Eqs. NS-num1, rk3), recovered from the GPU's projected velocity and pressure
    as u* = u^k + 2 alpha dt grad(p^k - p^{k-1}) (Eqs. NS-num2/3 with
    p^k = p^{k-1} + psi), at every face of each window's interior.
For the two-phase drop (AB2) the level set phi^{n+1} is compared at every cell with
the oracle's level-set update of the full fields, and B^{n+1} and u* on windows as
above.  The projection itself is a global solve; it is checked through a property
that holds at any size: the discrete divergence of u^k, in FP64 on the host from the stored
FP32 fields, is at the FP32 rounding level of the velocity.  Together with the u*
check, u^k - u* is then a discrete gradient that removes the divergence of u*.

Inputs: the benchmark's velocity recipe for each workload, a random pressure and a
large-deformation SPD conformation B = s (I + a S)^2 in place of B = I, so that the
advection, the upper-convected terms and (Saramito) both sides of the yield
surface are exercised from the first substep.  Tolerance: 1e-5 relative per field
(FP32 path, per step), as in the small-size tests.
"""

import numpy as np
import pytest

import oracle
from paper_1803_09563_gb300 import inputs
from oracle_windows import cut, predictor

pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)


def rd(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def run_first_substep(evp, grid, model, params, U, V, W, p, B, dt):
    sim = evp.Simulation(grid, model, params)
    evp.evp_set_graph(sim.handle, True)
    sim.set_state(U, V, W, p, B)
    sim.substep(dt, 0)
    code, bits, maxdiv = sim.sync()
    out = [sim.get(f).astype(np.float64) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P)]
    Bn = [sim.get(evp.EVP_BXX + c).astype(np.float64) for c in range(6)]
    sim.close()
    return out, Bn, maxdiv


def check_windows(g, prm, dt, force, state0, out, Bn, starts_list, widths, tol=1e-5):
    """Compare B^1 and the recovered u* with the oracle on each window; returns the
    window B^0 of the compared cells (for coverage checks)."""
    U, V, W, p, B = state0
    U1, V1, W1, p1 = out
    coef = 2.0 * oracle.RK3_ALPHA[0] * dt
    gp = oracle.grad_p(p1 - p, g)
    star_gpu = (U1 + coef * gp[0], V1 + coef * gp[1], W1 + coef * gp[2])
    seen = []
    worst = {'u*': 0.0, 'B': 0.0}
    for starts in starts_list:
        idx, star_o, Bn_o, B0_w = predictor(g, prm, dt, 0, U, V, W, p, B, starts, widths, force)
        for q in range(3):
            got = cut(star_gpu[q], starts, widths)[idx]
            ref = star_o[q][idx]
            err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
            assert err < tol, ('u*', q, starts, err)
            worst['u*'] = max(worst['u*'], err)
        for c in range(6):
            got = cut(Bn[c], starts, widths)[idx]
            ref = Bn_o[c][idx]
            err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
            assert err < tol, ('B', c, starts, err)
            worst['B'] = max(worst['B'], err)
        seen.append([b[idx] for b in B0_w])
    print('max relative error over the windows:', worst)
    return seen


def divergence_bound(g, U, V, W):
    """FP32 rounding of a face velocity moves the discrete divergence of a cell by at
    most eps32 |u|_max (1/dx + 1/dy + 1/dz)."""
    umax = max(np.abs(U).max(), np.abs(V).max(), np.abs(W).max())
    return EPS32 * umax * (1.0 / g.dx + 1.0 / g.dy + 1.0 / g.dz)


def test_saramito_channel_256x128x128_first_substep(evp):
    """Saramito EVP channel, 256x128x128, walls at y = +-1, Re 100, Wi 1, Bi 0.5,
    beta 0.5, the Poiseuille body force 2/Re, dt 2e-3: the benchmark workload."""
    nx, ny, nz = 256, 128, 128
    lx, ly, lz = 4 * np.pi, 2.0, 2 * np.pi
    Re, Wi, Bi, beta, dt = 100.0, 1.0, 0.5, 0.5, 2e-3
    geo = inputs.geometry(nx, ny, nz, lx, ly, lz, True)
    U, V, W = inputs.poiseuille(geo)
    u2, v2, w2 = inputs.scale_max(*inputs.random_solenoidal(geo, 1, 8), 1e-2)
    U, V, W = rd(U + u2), rd(v2), rd(w2)
    V[:, -1] = 0.0
    B = [rd(b) for b in inputs.spd_conformation(geo, 7, 0.6, scale=3.0)]
    p = rd(np.random.default_rng(9).standard_normal((nz, ny, nx)) * 0.05)
    grid = evp.make_grid(nx, ny, nz, lx, ly, lz, True)
    params = evp.make_params(Re=Re, Wi=Wi, beta=beta, Bi=Bi, dpdx=2.0 / Re, precision=evp.EVP_FP32)
    out, Bn, maxdiv = run_first_substep(evp, grid, 'saramito', params, U, V, W, p, B, dt)

    g = oracle.Grid(nx, ny, nz, lx, ly, lz, True)
    prm = oracle.Params.from_groups('saramito', Re, Wi, beta, Bi=Bi)
    force = (2.0 / Re, 0.0, 0.0)
    # windows across the periodic seams in x and in z, and one inside
    starts = [(244, 0, 50), (100, 0, 116), (17, 0, 3)]
    seen = check_windows(g, prm, dt, force, (U, V, W, p, B), out, Bn, starts, (24, None, 24))
    # both sides of the yield surface were compared (F = 0 and F > 0 of Table 1)
    F = np.concatenate([np.ravel(oracle.closure(b0, prm)[0]) for b0 in seen])
    assert (F == 0.0).sum() > 1000 and (F > 0.0).sum() > 1000
    # projection: the FP64 divergence of the stored FP32 velocity, and the GPU's own
    # FP64 residual of the same fields
    div = oracle.divergence(out[0], out[1], out[2], g)
    bound = divergence_bound(g, *out[:3])
    print('max|div u|:', np.abs(div).max(), 'GPU FP64 residual:', maxdiv, 'bound:', bound)
    assert np.abs(div).max() < bound
    assert maxdiv < bound
    assert abs(np.abs(div).max() - maxdiv) <= 1e-3 * bound + 1e-9 * maxdiv


def test_fene_p_turbulence_256cubed_first_substep(evp):
    """FENE-P forced turbulence, 256^3 periodic box 2 pi, Re 200, Wi 5, beta 0.9,
    L^2 900, ABC forcing A = 1 at k = 2, dt 1e-3: the benchmark workload."""
    n, L = 256, 2 * np.pi
    Re, Wi, beta, L2, dt = 200.0, 5.0, 0.9, 900.0, 1e-3
    A, kf = 1.0, 2.0
    geo = inputs.geometry(n, n, n, L, L, L)
    U, V, W = (rd(a) for a in inputs.scale_rms(*inputs.random_solenoidal(geo, 2, 16, spectrum='k-5/3',
                                                                          periodic_fft=True), 1.0))
    B = [rd(b) for b in inputs.spd_conformation(geo, 8, 0.5)]
    p = rd(np.random.default_rng(10).standard_normal((n, n, n)) * 0.1)
    grid = evp.make_grid(n, n, n, L, L, L)
    params = evp.make_params(Re=Re, Wi=Wi, beta=beta, L2=L2, abc_amp=A, abc_k=kf, precision=evp.EVP_FP32)
    out, Bn, maxdiv = run_first_substep(evp, grid, 'fene_p', params, U, V, W, p, B, dt)

    g = oracle.Grid(n, n, n, L, L, L)
    prm = oracle.Params.from_groups('fene_p', Re, Wi, beta, L2=L2)
    # the ABC force at the faces from its definition (each component is constant
    # along its own direction, so the centre coordinates are the face coordinates)
    xc, yc, zc = g.xc(), g.yc(), g.zc()
    shp = (n, n, n)
    force = (np.broadcast_to(A * (np.sin(kf * zc) + np.cos(kf * yc)), shp),
             np.broadcast_to(A * (np.sin(kf * xc) + np.cos(kf * zc)), shp),
             np.broadcast_to(A * (np.sin(kf * yc) + np.cos(kf * xc)), shp))
    starts = [(244, 250, 3), (100, 17, 240), (0, 128, 60)]
    check_windows(g, prm, dt, force, (U, V, W, p, B), out, Bn, starts, (24, 24, 24))
    div = oracle.divergence(out[0], out[1], out[2], g)
    bound = divergence_bound(g, *out[:3])
    print('max|div u|:', np.abs(div).max(), 'GPU FP64 residual:', maxdiv, 'bound:', bound)
    assert np.abs(div).max() < bound
    assert maxdiv < bound


def test_evp_drop_128x256x128_first_step(evp):
    """Two-phase buoyancy-driven drop in a Saramito fluid, 128x256x128 periodic box
    4 x 8 x 4, FP32, AB2 with the level set: drop of radius 0.5 at (2, 2, 2), Heaviside
    over 1.5 cells, Re 10, Wi 1, Bi 0.2 (tau_y = Bi), beta 0.5, viscosity ratio 1,
    surface tension 0.1 and drho g = 1 (Bond 10), re-distancing every 10 steps,
    dt 1e-3: the benchmark workload, one step from a moving, stressed state.

    * phi^{n+1} (Sec. 3.2.1: TVD-RK3 + WENO5 advection) at every cell, against the
      oracle's level-set update on the full fields;
    * B^{n+1} (Eq. ab2tau) and u* (Eq. ab2 with the CSF force and buoyancy),
      recovered as u^{n+1} + dt grad p^{n+1} (Eq. projection), on windows across the
      drop's interface and across the periodic seams;
    * the divergence of u^{n+1} at the FP32 rounding level."""
    from oracle.ab2 import TwoPhase, ab2_levelset
    from oracle import levelset as ls
    from oracle_windows import ab2_predictor
    nx, ny, nz = 128, 256, 128
    lx, ly, lz = 4.0, 8.0, 4.0
    dt = 1e-3
    geo = inputs.geometry(nx, ny, nz, lx, ly, lz)
    phi = rd(inputs.sphere_distance(geo, (2.0, 2.0, 2.0), 0.5))
    U, V, W = (rd(a) for a in inputs.scale_max(*inputs.random_solenoidal(geo, 3, 4), 0.5))
    B = [rd(b) for b in inputs.spd_conformation(geo, 11, 0.6, scale=12.0)]
    params = evp.make_params(Re=10.0, Wi=1.0, beta=0.5, Bi=0.2, bi_def=1, precision=evp.EVP_FP32,
                             integrator=evp.EVP_AB2, mu_ratio=1.0, ls_eps_cells=1.5, sigma=0.1, drho_g=1.0,
                             reinit_every=10, reinit_iters=2)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, lx, ly, lz), 'saramito', params)
    sim.set_state(U, V, W, None, B)
    sim.set(evp.EVP_PHI, phi)
    sim.step(dt)
    code, bits, maxdiv = sim.sync()
    U1, V1, W1, p1, phi1 = (sim.get(f).astype(np.float64)
                            for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P, evp.EVP_PHI))
    Bn = [sim.get(evp.EVP_BXX + c).astype(np.float64) for c in range(6)]
    sim.close()

    g = oracle.Grid(nx, ny, nz, lx, ly, lz)
    tp = TwoPhase('saramito', Re=10.0, Wi=1.0, beta=0.5, tau_y=0.2, mu_ratio=1.0, eps_cells=1.5, sigma=0.1,
                  drho_g=1.0, reinit_every=10, reinit_iters=2)
    st = oracle.State.rest(g, U, V, W)
    st.B = B
    phi1_o = ab2_levelset(phi, st, dt, g, tp, 0)
    err_phi = np.abs(phi1 - phi1_o).max() / np.abs(phi1_o).max()
    assert err_phi < 1e-5
    worst = {'phi': err_phi, 'u*': 0.0, 'B': 0.0}

    gp = oracle.grad_p(p1, g)
    star_gpu = (U1 + dt * gp[0], V1 + dt * gp[1], W1 + dt * gp[2])
    widths = (24, 24, 24)
    band = yielded = unyielded = 0
    eps = tp.eps_cells * g.dx
    # across the drop's lower interface (y = 1.5), its side (x = 2.5), and the seams
    for starts in ((52, 36, 52), (68, 52, 52), (120, 250, 120)):
        idx, star_o, Bn_o, B0_w, phw = ab2_predictor(g, tp, dt, U, V, W, np.zeros_like(U), B, phi1_o, starts,
                                                     widths)
        for q in range(3):
            got = cut(star_gpu[q], starts, widths)[idx]
            ref = star_o[q][idx]
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err < 1e-5, ('u*', q, starts, err)
            worst['u*'] = max(worst['u*'], err)
        for c in range(6):
            got = cut(Bn[c], starts, widths)[idx]
            ref = Bn_o[c][idx]
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err < 1e-5, ('B', c, starts, err)
            worst['B'] = max(worst['B'], err)
        H = ls.heaviside(phw[idx], eps)
        band += ((H > 0.01) & (H < 0.99)).sum()
        mu_s, mu_p = tp.mixture(H)
        F = oracle.closure([b[idx] for b in B0_w],
                           oracle.Params('saramito', mu_s=mu_s, mu_p=mu_p, lam=tp.Wi, tau_y=tp.tau_y))[0]
        yielded += ((F > 0.0) & (H > 0.99)).sum()
        unyielded += ((F == 0.0) & (H > 0.99)).sum()
    # the interface band and both sides of the yield surface were compared
    assert band > 100 and yielded > 50 and unyielded > 50
    div = oracle.divergence(U1, V1, W1, g)
    bound = divergence_bound(g, U1, V1, W1)
    print('max relative error:', worst, 'band/yielded/unyielded cells:', band, yielded, unyielded)
    print('max|div u|:', np.abs(div).max(), 'GPU FP64 residual:', maxdiv, 'bound:', bound)
    assert np.abs(div).max() < bound
    assert maxdiv < bound


def test_saramito_channel_graph_replay_equals_direct_launches(evp):
    """The benchmark's own launch path at its own size: the channel workload exactly
    as the benchmark sets it up (velocity recipe, B = I, a torch stream), two RK3
    steps replayed from the captured step graphs (one per B buffer parity) against
    the same steps launched directly, all fields bit for bit.  The windows above
    check the direct launches against the oracle."""
    import torch
    nx, ny, nz = 256, 128, 128
    lx, ly, lz = 4 * np.pi, 2.0, 2 * np.pi
    Re, dt = 100.0, 2e-3
    geo = inputs.geometry(nx, ny, nz, lx, ly, lz, True)
    U, V, W = inputs.poiseuille(geo)
    u2, v2, w2 = inputs.scale_max(*inputs.random_solenoidal(geo, 1, 8), 1e-2)
    U, V, W = U + u2, v2, w2
    names = [evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P] + [evp.EVP_BXX + c for c in range(6)]
    out = []
    for graph in (True, False):
        stream = torch.cuda.Stream()
        sim = evp.Simulation(evp.make_grid(nx, ny, nz, lx, ly, lz, True), 'saramito',
                             evp.make_params(Re=Re, Wi=1.0, beta=0.5, Bi=0.5, dpdx=2.0 / Re,
                                             precision=evp.EVP_FP32), stream=stream.cuda_stream)
        sim.set_state(U, V, W)
        evp.evp_set_graph(sim.handle, graph)
        for _ in range(3):
            sim.step(dt)
        sim.sync()
        out.append([sim.get(f) for f in names])
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
