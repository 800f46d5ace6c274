"""Pins the sampled-parity method of the full-size GPU tests: the oracle's substep
predictor (u*, B^k) on a window cut from the full fields equals, at every cell at
least MARGIN cells from the window's cut faces, the predictor on the full fields,
bit for bit; cells on the cut faces differ (the window's own periodic wrap reaches
them), so the comparison region is not vacuous."""

import numpy as np
import pytest

import oracle
from paper_1803_09563_gb300 import inputs
from oracle_windows import MARGIN, cut, predictor


def full_case(shape, walls, model, extra, seed):
    nx, ny, nz = shape
    ly = 2.0 if walls else 2 * np.pi
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, seed, 3), 1.0)
    if walls:
        U = U + inputs.poiseuille(geo)[0]
        V[:, -1] = 0.0
    B = inputs.spd_conformation(geo, seed + 1, 0.6)
    p = np.random.default_rng(seed + 2).standard_normal((nz, ny, nx)) * 0.1
    g = oracle.Grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls)
    prm = oracle.Params.from_groups(model, Re=2.0, Wi=0.8, beta=0.4, **extra)
    return g, prm, U, V, W, p, B


@pytest.mark.parametrize("walls,model,extra", [(True, 'saramito', {'Bi': 0.4}), (False, 'fene_p', {'L2': 60.0})])
def test_window_interior_equals_full_predictor(walls, model, extra):
    shape = (40, 24, 36)
    g, prm, U, V, W, p, B = full_case(shape, walls, model, extra, 5)
    dt = 2e-3
    force = (0.3, 0.0, 0.1)
    st = oracle.State.rest(g, U, V, W)
    st.p = p
    st.B = B
    star, Bn = oracle.rk3_substep(st, 0, dt, g, prm, force, predictor_only=True)
    widths = (24, None, 24) if walls else (24, 24, 24)
    for starts in ((30, 0, 20), (5, 13, 0)):
        idx, star_w, Bn_w, _ = predictor(g, prm, dt, 0, U, V, W, p, B, starts, widths, force)
        for full, win in zip(list(star) + list(Bn), list(star_w) + list(Bn_w)):
            ref = cut(full, starts, widths)
            assert np.array_equal(win[idx], ref[idx])
            # the cut faces themselves see the window's wrap, not the full field
            assert not np.array_equal(win[:, :, :1], ref[:, :, :1])
    assert MARGIN * 2 < 24


@pytest.mark.parametrize("walls", [True, False])
def test_predictor_recovered_from_projected_fields(walls):
    """The full-size GPU tests recover u* from the projected velocity and pressure as
    u^k + 2 alpha dt grad(p^k - p^{k-1}) (Eqs. NS-num2/3 with p^k = p^{k-1} + psi).
    On the oracle's own substep this recovers its predictor to rounding, the wall
    face included, and the projected velocity is divergence-free."""
    g, prm, U, V, W, p, B = full_case((32, 16, 24), walls, 'saramito', {'Bi': 0.4}, 9)
    dt = 2e-3
    st = oracle.State.rest(g, U, V, W)
    st.p = p
    st.B = B
    star, _ = oracle.rk3_substep(st, 0, dt, g, prm, (0.3, 0.0, 0.0), predictor_only=True)
    s1 = oracle.rk3_substep(st, 0, dt, g, prm, (0.3, 0.0, 0.0))
    coef = 2.0 * oracle.RK3_ALPHA[0] * dt
    gp = oracle.grad_p(s1.p - p, g)
    for q, vel in enumerate((s1.U, s1.V, s1.W)):
        assert np.abs(vel + coef * gp[q] - star[q]).max() < 1e-12 * np.abs(star[q]).max() + 1e-15
    assert np.abs(oracle.divergence(s1.U, s1.V, s1.W, g)).max() < 1e-11


def test_ab2_window_interior_equals_full_predictor():
    """The same for the two-phase AB2 predictor (mixture properties from H(phi^{n+1}),
    CSF force and buoyancy, stress and momentum), phi^{n+1} taken from the full
    fields."""
    from oracle.ab2 import TwoPhase, ab2_levelset, ab2_predictor as full_predictor
    from oracle_windows import ab2_predictor
    nx, ny, nz = 40, 48, 36
    geo = inputs.geometry(nx, ny, nz, 1.25, 1.5, 1.125)
    g = oracle.Grid(nx, ny, nz, 1.25, 1.5, 1.125)
    phi = inputs.sphere_distance(geo, (0.6, 0.7, 0.55), 0.3)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, 4, 3), 0.5)
    B = inputs.spd_conformation(geo, 6, 0.6, scale=5.0)
    p = np.random.default_rng(8).standard_normal((nz, ny, nx)) * 0.1
    tp = TwoPhase('saramito', Re=10.0, Wi=1.0, beta=0.5, tau_y=0.2, mu_ratio=0.5, sigma=0.1, drho_g=1.0)
    st = oracle.State.rest(g, U, V, W)
    st.p = p
    st.B = B
    dt = 1e-3
    phi1 = ab2_levelset(phi, st, dt, g, tp, 0)
    star, Bn, _, _, _ = full_predictor(st, phi1, dt, g, tp, 0)
    widths = (24, 24, 24)
    band = 0
    # one window across the drop's interface (x = 0.9), one across the periodic seams
    for starts in ((18, 10, 6), (30, 40, 25)):
        idx, star_w, Bn_w, _, phw = ab2_predictor(g, tp, dt, U, V, W, p, B, phi1, starts, widths)
        band += (np.abs(phw[idx]) < 1.5 * g.dx).sum()
        for full, win in zip(list(star) + list(Bn), list(star_w) + list(Bn_w)):
            ref = cut(full, starts, widths)
            assert np.array_equal(win[idx], ref[idx])
            assert not np.array_equal(win[:, :, :1], ref[:, :, :1])
    assert band > 0


def test_spd_conformation_is_symmetric_positive_definite():
    """The large-deformation input B = s (I + a S)^2 is positive definite (its
    eigenvalues are s times the squares of those of I + a S) and its deviator
    scales with s."""
    geo = inputs.geometry(16, 12, 10, 2 * np.pi, 2.0, 2 * np.pi, True)
    B = inputs.spd_conformation(geo, 7, 0.6, scale=3.0)
    M = np.stack([np.stack([B[0], B[1], B[2]], -1), np.stack([B[1], B[3], B[4]], -1),
                  np.stack([B[2], B[4], B[5]], -1)], -2)
    assert np.linalg.eigvalsh(M).min() > 0.0
    B1 = inputs.spd_conformation(geo, 7, 0.6, scale=1.0)
    for c in range(6):
        assert np.allclose(B[c], 3.0 * B1[c], rtol=1e-15, atol=0.0)
    S = inputs.random_conformation(geo, 7, amp=1.0)
    m = [(1.0 if c in (0, 3, 5) else 0.0) + 0.6 * (S[c] - (1.0 if c in (0, 3, 5) else 0.0)) for c in range(6)]
    Mm = np.stack([np.stack([m[0], m[1], m[2]], -1), np.stack([m[1], m[3], m[4]], -1),
                   np.stack([m[2], m[4], m[5]], -1)], -2)
    sq = Mm @ Mm
    assert np.allclose(M, 3.0 * sq, rtol=1e-14, atol=1e-14)
