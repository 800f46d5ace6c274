"""Pins for the oracle's monitoring quantities (``oracle/diagnostics.py``):
closed forms of single Fourier modes, the steady simple-shear conformation, the
Saramito plug edge of Sec. 4.1.1, a library determinant, and planted slips."""

import numpy as np
import pytest

from oracle.grid import Grid
from oracle.models import Params
from oracle import diagnostics as dg


def _prm(model, tau_y=0.0, L2=0.0, mu_p=0.5, lam=2.0):
    return Params(model, mu_s=0.5, mu_p=mu_p, lam=lam, tau_y=tau_y, L2=L2)


def _identity(g):
    one, zero = np.ones(g.shape), np.zeros(g.shape)
    return [one.copy(), zero.copy(), zero.copy(), one.copy(), zero.copy(), one.copy()]


def test_kinetic_energy_of_fourier_modes():
    """u = a sin(2 pi y/ly), v = b cos(2 pi z/lz), w = c on a periodic box: the
    discrete sums of sin^2 and cos^2 over a whole period are N/2 (N >= 3), so
    E = 1/2 V (a^2/2 + b^2/2 + c^2) exactly up to rounding."""
    g = Grid(12, 16, 8, 1.5, 2.0, 3.0)
    a, b, c = 0.7, -1.3, 0.4
    U = a * np.sin(2 * np.pi * g.yc() / g.ly) * np.ones(g.shape)
    V = b * np.cos(2 * np.pi * g.zc() / g.lz) * np.ones(g.shape)
    W = c * np.ones(g.shape)
    got = dg.diagnostics(U, V, W, None, g, _prm('newtonian'))
    vol = g.lx * g.ly * g.lz
    assert got['kinetic_energy'] == pytest.approx(0.5 * vol * (a * a / 2 + b * b / 2 + c * c), rel=1e-14)
    assert got['min_det_B'] == np.inf and got['yielded_cells'] == 0 and got['nonfinite_cells'] == 0
    # u varies in y only, v in z only and w is uniform: du/dx = dv/dy = dw/dz = 0
    assert got['max_div'] == pytest.approx(0.0, abs=1e-12)


def test_det_of_the_steady_shear_conformation():
    """Oldroyd-B steady simple shear (Sec. 4.1.3): B_xx = 1 + 2 Wi^2, B_xy = Wi,
    B_yy = B_zz = 1 for the Weissenberg number Wi = lambda gdot, so that
    det B = 1 + Wi^2 and tr B = 3 + 2 Wi^2."""
    g = Grid(4, 6, 5, 1.0, 1.0, 1.0)
    wi = np.linspace(0.0, 3.0, g.ny)[None, :, None] * np.ones(g.shape)
    B = _identity(g)
    B[0] = 1 + 2 * wi ** 2
    B[1] = wi.copy()
    assert np.allclose(dg.det3_sym(B), 1 + wi ** 2, rtol=1e-14, atol=0)
    z = np.zeros(g.shape)
    got = dg.diagnostics(z, z, z, B, g, _prm('oldroyd_b'))
    assert got['min_det_B'] == pytest.approx(1.0, abs=1e-15)
    assert got['max_tr_B'] == pytest.approx(3 + 2 * 9.0, rel=1e-15)
    assert got['yielded_fraction'] == 1.0


def test_det_matches_the_library_and_is_rotation_invariant():
    rng = np.random.default_rng(11)
    for _ in range(30):
        A = rng.standard_normal((3, 3))
        M = A @ A.T + 0.1 * np.eye(3) if rng.random() < 0.5 else A + A.T
        B = [M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]]
        assert dg.det3_sym(B) == pytest.approx(np.linalg.det(M), rel=1e-12, abs=1e-12)
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        R = Q @ M @ Q.T
        BR = [R[0, 0], R[0, 1], R[0, 2], R[1, 1], R[1, 2], R[2, 2]]
        assert dg.det3_sym(BR) == pytest.approx(dg.det3_sym(B), rel=1e-10, abs=1e-12)


def test_deviatoric_magnitude_closed_forms():
    """Pure shear tau_xy = s gives |tau^d| = |s|; tau = diag(s, -s, 0) (already
    deviatoric) gives |tau^d| = |s|; an isotropic tau = p I has no deviator."""
    s, p, gm = 0.37, 5.0, 0.25
    one, zero = 1.0, 0.0
    shear = [one, s / gm, zero, one, zero, one]
    assert dg.deviatoric_magnitude(shear, gm) == pytest.approx(s, rel=1e-15)
    normal = [one + s / gm, zero, zero, one - s / gm, zero, one]
    assert dg.deviatoric_magnitude(normal, gm) == pytest.approx(s, rel=1e-14)
    iso = [one + p / gm, zero, zero, one + p / gm, zero, one + p / gm]
    assert dg.deviatoric_magnitude(iso, gm) == pytest.approx(0.0, abs=1e-14)


def saramito_shear_conformation(g, G, mu_p, lam):
    """B of the steady yielded Saramito simple shear in a channel: tau_xy = -G y
    (the momentum balance), tau_xx = 2 lam tau_xy^2 / mu_p, tau_yy = tau_zz = 0
    (Table 1 with F = a in steady shear), B = I + tau lam / mu_p."""
    y = g.yc() * np.ones(g.shape)
    txy = -G * y
    txx = 2 * lam * txy ** 2 / mu_p
    B = _identity(g)
    B[0] = 1 + txx * lam / mu_p
    B[1] = txy * lam / mu_p
    return B


def test_yielded_cells_follow_the_plug_edge_of_the_channel():
    """The yield surface of the steady Saramito channel sits at |y| = y0 with
    (G y0)^2 = 3 mu_p^2 (-1 + sqrt(1 + 16 lam^2 tau_y^2 / (3 mu_p^2))) / (8 lam^2):
    there |tau^d|^2 = tau_xy^2 + tau_xx^2/3 = tau_y^2.  On the shear conformation
    of that channel the yielded cells are exactly the cell centres with |y| > y0."""
    mu_p, lam, tau_y, G = 0.6, 0.8, 0.5 * 1.25 ** -1, 1.0
    y0 = np.sqrt(3 * mu_p ** 2 * (-1 + np.sqrt(1 + 16 * lam ** 2 * tau_y ** 2 / (3 * mu_p ** 2)))
                 / (8 * lam ** 2)) / G
    for ny in (32, 50, 96):
        g = Grid(3, ny, 2, 1.0, 2.0, 1.0, walls_y=True)
        B = saramito_shear_conformation(g, G, mu_p, lam)
        z = np.zeros(g.shape)
        got = dg.diagnostics(z, z, z, B, g, _prm('saramito', tau_y=tau_y, mu_p=mu_p, lam=lam))
        yc = g.yc().ravel()
        expect = int(np.count_nonzero(np.abs(yc) > y0)) * g.nx * g.nz
        assert got['yielded_cells'] == expect
        assert 0 < expect < g.ncells
        # the plug edge is inside the channel, and a plug of width ~ 2 y0 is not yielded
        assert got['yielded_fraction'] == pytest.approx(1 - 2 * y0 / g.ly, abs=2.0 / ny)


def test_yield_limits_and_models_without_a_yield_surface():
    g = Grid(4, 8, 4, 1.0, 2.0, 1.0, walls_y=True)
    B = saramito_shear_conformation(g, 1.0, 0.6, 0.8)
    z = np.zeros(g.shape)
    assert dg.diagnostics(z, z, z, B, g, _prm('saramito', tau_y=0.0))['yielded_cells'] == g.ncells
    assert dg.diagnostics(z, z, z, B, g, _prm('saramito', tau_y=1e9))['yielded_cells'] == 0
    assert dg.diagnostics(z, z, z, B, g, _prm('neo_hookean'))['yielded_cells'] == 0
    fene = dg.diagnostics(z, z, z, B, g, _prm('fene_p', L2=100.0))
    assert fene['yielded_cells'] == g.ncells
    assert fene['max_tr_B_over_L2'] == pytest.approx(fene['max_tr_B'] / 100.0, rel=1e-15)


def test_brute_force_on_a_tiny_state():
    """Every quantity recomputed with scalar loops over a 3 x 4 x 2 state."""
    rng = np.random.default_rng(5)
    g = Grid(3, 4, 2, 0.9, 1.1, 0.7, walls_y=True)
    U, V, W = (rng.standard_normal(g.shape) for _ in range(3))
    V[:, -1, :] = 0.0                       # top wall face
    B = [rng.standard_normal(g.shape) * 0.3 + (1.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    prm = _prm('fene_p', L2=20.0)
    got = dg.diagnostics(U, V, W, B, g, prm)
    ke, dets, trs, dmax = 0.0, [], [], 0.0
    for k in range(g.nz):
        for j in range(g.ny):
            for i in range(g.nx):
                ke += U[k, j, i] ** 2 + V[k, j, i] ** 2 + W[k, j, i] ** 2
                M = np.array([[B[0][k, j, i], B[1][k, j, i], B[2][k, j, i]],
                              [B[1][k, j, i], B[3][k, j, i], B[4][k, j, i]],
                              [B[2][k, j, i], B[4][k, j, i], B[5][k, j, i]]])
                dets.append(np.linalg.det(M))
                trs.append(np.trace(M))
                um = U[k, j, i - 1]
                vm = V[k, j - 1, i] if j > 0 else 0.0
                wm = W[k - 1, j, i]
                d = (U[k, j, i] - um) / g.dx + (V[k, j, i] - vm) / g.dy + (W[k, j, i] - wm) / g.dz
                dmax = max(dmax, abs(d))
    assert got['kinetic_energy'] == pytest.approx(0.5 * g.dx * g.dy * g.dz * ke, rel=1e-14)
    assert got['min_det_B'] == pytest.approx(min(dets), rel=1e-12)
    assert got['max_tr_B'] == pytest.approx(max(trs), rel=1e-14)
    assert got['max_tr_B_over_L2'] == pytest.approx(max(trs) / 20.0, rel=1e-14)
    assert got['max_div'] == pytest.approx(dmax, rel=1e-13)


def test_nonfinite_cells_are_counted_once_per_cell():
    g = Grid(4, 4, 4, 1.0, 1.0, 1.0)
    z = np.zeros(g.shape)
    U, V, W = z.copy(), z.copy(), z.copy()
    B = _identity(g)
    U[1, 2, 3] = np.nan
    B[4][0, 0, 0] = np.inf
    W[3, 3, 3] = -np.inf
    B[0][3, 3, 3] = np.nan                  # same cell as the W entry
    got = dg.diagnostics(U, V, W, B, g, _prm('oldroyd_b'))
    assert got['nonfinite_cells'] == 3


@pytest.mark.parametrize('slip', ['half', 'sign', 'trace'])
def test_planted_slips_fail(monkeypatch, slip):
    """A dropped 1/2 in the energy, a cofactor sign or a dropped deviatoric
    trace each break one of the pins above."""
    if slip == 'half':
        orig = dg.diagnostics

        def wrong(U, V, W, B, g, prm):
            out = orig(U, V, W, B, g, prm)
            out['kinetic_energy'] *= 2
            return out
        monkeypatch.setattr(dg, 'diagnostics', wrong)
        with pytest.raises(AssertionError):
            test_kinetic_energy_of_fourier_modes()
    elif slip == 'sign':
        def wrong(B):
            xx, xy, xz, yy, yz, zz = B
            return xx * (yy * zz - yz * yz) + xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz)
        monkeypatch.setattr(dg, 'det3_sym', wrong)
        with pytest.raises(AssertionError):
            test_det_of_the_steady_shear_conformation()
    else:
        def wrong(B, g_mod):
            t = [g_mod * (B[c] - (1.0 if c in (0, 3, 5) else 0.0)) for c in range(6)]
            return np.sqrt(0.5 * (t[0] * t[0] + t[3] * t[3] + t[5] * t[5]) + t[1] * t[1] + t[2] * t[2] + t[4] * t[4])
        monkeypatch.setattr(dg, 'deviatoric_magnitude', wrong)
        with pytest.raises(AssertionError):
            test_yielded_cells_follow_the_plug_edge_of_the_channel()
