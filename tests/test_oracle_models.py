"""Pins for the oracle's constitutive closures (Table 1) and the source part of
Eq. SRM2, through homogeneous-shear closed forms (Sec. 4.1.3) and brute force."""

import os

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from oracle.models import ucd_terms, rt_local, closure, tau_from_B, Params, COMP_IJ

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def sym(B6):
    M = np.zeros((3, 3))
    for c, (a, b) in enumerate(COMP_IJ):
        M[a, b] = M[b, a] = B6[c]
    return M


def test_ucd_terms_brute_force():
    """L B + B L^T written out per component equals the 3x3 matrix products."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        B6 = rng.standard_normal(6)
        L = rng.standard_normal((3, 3))
        got = ucd_terms(list(B6), [[L[i, j] for j in range(3)] for i in range(3)])
        ref = L @ sym(B6) + sym(B6) @ L.T
        for c, (a, b) in enumerate(COMP_IJ):
            assert abs(got[c] - ref[a, b]) < 1e-13


def integrate_homogeneous(prm, Lfun, t_end, dt):
    """Integrate dB/dt = rt_local(B, L(t)) (uniform field, no advection) with the
    paper's low-storage RK3 constants (Eq. RK); returns times and B history."""
    B = [np.array(1.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    hist = None
    t = 0.0
    ts, Bs = [0.0], [list(B)]
    nsteps = int(round(t_end / dt))
    for _ in range(nsteps):
        tk = t
        for k in range(3):
            a, z, x = oracle.RK3_ALPHA[k], oracle.RK3_ZETA[k], oracle.RK3_XI[k]
            L = Lfun(tk)
            rt = rt_local(B, L, prm)
            B = [B[c] + dt * (z * rt[c] + (x * hist[c] if x != 0.0 else 0.0)) for c in range(6)]
            hist = rt
            tk += 2.0 * a * dt
        t += dt
        ts.append(t)
        Bs.append(list(B))
    return np.array(ts), Bs


def shear_L(gdot):
    return lambda t: [[0.0, gdot, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]


def test_oldroyd_b_startup_shear_closed_form():
    """tau_xy = mu_p gdot (1 - e^{-t/lam}), tau_xx = 2 mu_p lam gdot^2 [1 - e^{-t/lam}(1 + t/lam)],
    tau_yy = 0 (Eq. SRM2 with the Oldroyd-B row of Table 1), and the steady values
    tau_xy = mu_p gdot, N1 = 2 mu_p lam gdot^2."""
    prm = Params.from_groups('oldroyd_b', Re=1.0, Wi=0.7, beta=0.3)
    gdot = 1.3
    ts, Bs = integrate_homogeneous(prm, shear_L(gdot), 12.0, 2e-3)
    mu_p, lam = prm.mu_p, prm.lam
    for t_check in (0.5, 2.0, 12.0):
        n = int(round(t_check / 2e-3))
        tau = tau_from_B(Bs[n], prm)
        e = np.exp(-t_check / lam)
        assert abs(tau[1] - mu_p * gdot * (1 - e)) < 1e-8
        assert abs(tau[0] - 2 * mu_p * lam * gdot ** 2 * (1 - e * (1 + t_check / lam))) < 1e-8
        assert abs(tau[3]) < 1e-12 and abs(tau[5]) < 1e-12
    tau = tau_from_B(Bs[-1], prm)
    assert abs(tau[1] - mu_p * gdot) < 1e-6
    assert abs((tau[0] - tau[3]) - 2 * mu_p * lam * gdot ** 2) < 1e-5


def saramito_yield_time(mu_p, lam, gdot, tau_y):
    """Pre-yield (F = 0) closed form: tau_xy = (mu_p/lam) gdot t, tau_xx = (mu_p/lam) (gdot t)^2;
    yield when tau_xy^2 + tau_xx^2/3 = tau_y^2."""
    g = mu_p / lam
    f = lambda t: (g * gdot * t) ** 2 + (g * (gdot * t) ** 2) ** 2 / 3.0 - tau_y ** 2
    return brentq(f, 1e-9, 1e3)


def test_saramito_startup_shear_yield_time_matches_paper():
    """Sec. 4.1.3 (Fig. uncoupl a): Wi = 1, Bi = 1, beta = 1/9 start-up shear yields
    at T ~ 1.  The closed form gives 0.97929; the oracle's stress stays on the
    pre-yield closed form until then and F turns positive within one step of it."""
    gold = dict(l.split('=') for l in open(os.path.join(GOLDEN, 'saramito_startup.txt')).read().split()
                if '=' in l)
    prm = Params.from_groups('saramito', Re=1.0, Wi=1.0, beta=1.0 / 9.0, Bi=1.0)
    ty = saramito_yield_time(prm.mu_p, prm.lam, 1.0, prm.tau_y)
    assert abs(ty - float(gold['closed_form_yield_time'])) < 1e-4
    assert abs(ty - float(gold['paper_yield_time'])) < float(gold['paper_tolerance'])
    dt = 1e-3
    ts, Bs = integrate_homogeneous(prm, shear_L(1.0), 1.5, dt)
    g = prm.mu_p / prm.lam
    yielded = None
    for t, B in zip(ts, Bs):
        F, _ = closure(B, prm)
        if F > 0 and yielded is None:
            yielded = t
        if t < ty - dt:
            tau = tau_from_B(B, prm)
            assert abs(tau[1] - g * t) < 1e-10
            assert abs(tau[0] - g * t * t) < 1e-10
    assert abs(yielded - ty) <= 2 * dt


def test_saramito_yielded_steady_shear():
    """Steady yielded simple shear: B_yy = 1, tau_xy = mu_p gdot / F,
    tau_xx = 2 mu_p lam gdot^2 / F^2, with F = 1 - tau_y/|tau^d| and
    |tau^d|^2 = tau_xy^2 + tau_xx^2/3 (root found here independently)."""
    prm = Params.from_groups('saramito', Re=1.0, Wi=0.5, beta=0.2, Bi=0.3)
    gdot = 1.0
    mu_p, lam, ty = prm.mu_p, prm.lam, prm.tau_y

    def resid(F):
        txy = mu_p * gdot / F
        txx = 2 * mu_p * lam * gdot ** 2 / F ** 2
        return F - (1 - ty / np.sqrt(txy ** 2 + txx ** 2 / 3))
    F = brentq(resid, 1e-6, 1.0)
    ts, Bs = integrate_homogeneous(prm, shear_L(gdot), 25.0, 5e-3)
    tau = tau_from_B(Bs[-1], prm)
    assert abs(tau[1] - mu_p * gdot / F) < 1e-7
    assert abs(tau[0] - 2 * mu_p * lam * gdot ** 2 / F ** 2) < 1e-7


def test_saramito_bi_zero_is_oldroyd_b_bitwise():
    rng = np.random.default_rng(5)
    B = [np.eye(3)[a, b] + 0.3 * rng.standard_normal((4, 5)) for a, b in COMP_IJ]
    L = [[rng.standard_normal((4, 5)) for _ in range(3)] for _ in range(3)]
    ob = Params.from_groups('oldroyd_b', Re=2.0, Wi=0.8, beta=0.4)
    sa = Params.from_groups('saramito', Re=2.0, Wi=0.8, beta=0.4, Bi=0.0)
    r1, r2 = rt_local(B, L, ob), rt_local(B, L, sa)
    for c in range(6):
        np.testing.assert_array_equal(r1[c], r2[c])


def test_saramito_zero_stress_guard():
    """|tau^d| = 0: F = 0 when tau_y > 0, F = 1 when tau_y = 0 (Reading 7)."""
    B = [np.array(1.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    F, a = closure(B, Params.from_groups('saramito', 1.0, 1.0, 0.5, Bi=0.2))
    assert F == 0.0 and a == 0.0
    F, a = closure(B, Params.from_groups('saramito', 1.0, 1.0, 0.5, Bi=0.0))
    assert F == 1.0 and a == 1.0


FENE_P_SHEAR = dict(Re=1.0, Wi=0.6, beta=0.5, L2=50.0, gdot=2.0)


def fene_p_steady_shear_root():
    """Steady simple shear of FENE-P (Table 1, upper-convected B): B_yy = B_zz =
    a/F, B_xy = lam gdot B_yy / F, B_xx = (a + 2 lam gdot B_xy)/F with
    F = L^2/(L^2 - tr B), solved here by a scalar root find."""
    c = FENE_P_SHEAR
    prm = Params.from_groups('fene_p', Re=c['Re'], Wi=c['Wi'], beta=c['beta'], L2=c['L2'])
    gdot, lam, L2 = c['gdot'], prm.lam, prm.L2
    a = L2 / (L2 - 3.0)

    def parts(F):
        byy = a / F
        bxy = lam * gdot * byy / F
        bxx = (a + 2 * lam * gdot * bxy) / F
        return bxx, bxy, byy

    def resid(F):
        bxx, bxy, byy = parts(F)
        return F - L2 / (L2 - (bxx + 2 * byy))
    F = brentq(resid, 1.0 + 1e-9, 50.0)
    return prm, gdot, a, F, parts(F)


def fene_p_steady_shear_oracle():
    """The oracle's homogeneous shear integrated to steady state (Eq. RK weights)."""
    prm, gdot, _, _, _ = fene_p_steady_shear_root()
    ts, Bs = integrate_homogeneous(prm, shear_L(gdot), 20.0, 2e-3)
    return Bs[-1]


def test_fene_p_identity_fixed_point_and_steady_shear():
    """B = I is a fixed point at rest (F(I) = a); the oracle's homogeneous shear
    reaches the steady conformation of the root find."""
    prm, gdot, a, F, (bxx, bxy, byy) = fene_p_steady_shear_root()
    I6 = [np.array(1.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    Z = [[0.0] * 3 for _ in range(3)]
    assert max(abs(v) for v in rt_local(I6, Z, prm)) < 1e-15
    B = fene_p_steady_shear_oracle()
    assert abs(B[0] - bxx) < 1e-7 and abs(B[1] - bxy) < 1e-8 and abs(B[3] - byy) < 1e-9


def fene_p_stress_errors(B, tau_fn):
    """Errors of tau = tau_fn(B) against steady FENE-P shear: tau_yy = tau_zz = 0,
    tau_xy = mu_p gdot a / F and N1 = tau_xx - tau_yy = 2 mu_p lam gdot^2 a / F^2
    (from tau = (mu_p/lam)(F B - a I) and the steady balance F B - a I = lam (L B + B L^T)),
    F from the root find."""
    prm, gdot, a, F, _ = fene_p_steady_shear_root()
    tau = tau_fn(B, prm)
    mu_p, lam = prm.mu_p, prm.lam
    return {'tau_yy': abs(float(tau[3])), 'tau_zz': abs(float(tau[5])),
            'tau_xy': abs(float(tau[1]) - mu_p * gdot * a / F) / (mu_p * gdot),
            'N1': abs(float(tau[0] - tau[3]) - 2 * mu_p * lam * gdot ** 2 * a / F ** 2) / (mu_p * lam * gdot ** 2)}


def test_fene_p_stress_from_conformation_in_steady_shear():
    """The FENE-P branch of the stress-from-B inversion (Table 1): in steady simple
    shear the normal stresses tau_yy and tau_zz vanish, tau_xy = mu_p gdot a/F and
    N1 = 2 mu_p lam gdot^2 a/F^2, with F from the independent root find."""
    import oracle.models as om
    err = fene_p_stress_errors(fene_p_steady_shear_oracle(), om.tau_from_B)
    assert err['tau_yy'] < 1e-9 and err['tau_zz'] < 1e-9, err
    assert err['tau_xy'] < 1e-7 and err['N1'] < 1e-6, err


@pytest.mark.parametrize('plant', ['B_minus_aI', 'FB_minus_I', 'modulus_mu_p'])
def test_fene_p_stress_pin_catches_planted_mistakes(plant, monkeypatch):
    """Each plausible slip in the FENE-P inversion gives an isotropic or scaled
    error that the rest state cannot see; the steady-shear pin fails on each."""
    import oracle.models as om
    B = fene_p_steady_shear_oracle()
    diag = (True, False, False, True, False, True)

    def bad(B, prm):
        g = prm.mu_p / prm.lam
        F, a = om.closure(B, prm)
        if plant == 'B_minus_aI':
            return [g * (B[c] - (a if diag[c] else 0.0)) for c in range(6)]
        if plant == 'FB_minus_I':
            return [g * (F * B[c] - (1.0 if diag[c] else 0.0)) for c in range(6)]
        return [prm.mu_p * (F * B[c] - (a if diag[c] else 0.0)) for c in range(6)]
    monkeypatch.setattr(om, 'tau_from_B', bad)
    err = fene_p_stress_errors(B, om.tau_from_B)
    assert not (err['tau_yy'] < 1e-9 and err['tau_zz'] < 1e-9 and err['tau_xy'] < 1e-7 and err['N1'] < 1e-6), err


def test_fene_p_steady_shear_pin_catches_a_planted_closure_mistake(monkeypatch):
    """A slip in the FENE-P closure itself (a = 1 instead of L^2/(L^2 - 3)) moves the
    steady conformation away from the root find."""
    import oracle.models as om
    orig = om.closure

    def bad(B, prm):
        F, a = orig(B, prm)
        return (F, 1.0) if prm.model == 'fene_p' else (F, a)
    monkeypatch.setattr(om, 'closure', bad)
    _, _, _, _, (bxx, bxy, byy) = fene_p_steady_shear_root()
    B = fene_p_steady_shear_oracle()
    assert not (abs(B[0] - bxx) < 1e-7 and abs(B[1] - bxy) < 1e-8 and abs(B[3] - byy) < 1e-9)


def test_oldroyd_b_oscillatory_shear_maxwell_closed_form():
    """Sec. 4.1.3 oscillatory shear, Bi = 0, beta = 0 (Fig. uncoupl b): strain
    gamma0 sin(w t); tau_xy obeys lam dtau/dt + tau = mu_p gamma0 w cos(w t), so
    tau_xy = mu_p gamma0 w [cos wt + lam w sin wt - e^{-t/lam}] / (1 + (lam w)^2)."""
    w, g0 = 2.0, 0.7
    prm = Params.from_groups('saramito', Re=1.0, Wi=0.1 / w, beta=0.0, Bi=0.0)
    lam, mu_p = prm.lam, prm.mu_p
    Lf = lambda t: [[0.0, g0 * w * np.cos(w * t), 0.0], [0.0] * 3, [0.0] * 3]
    ts, Bs = integrate_homogeneous(prm, Lf, 6.0, 1e-3)
    for n in (500, 2000, 6000):
        t = ts[n]
        ref = mu_p * g0 * w * (np.cos(w * t) + lam * w * np.sin(w * t) - np.exp(-t / lam)) / (1 + (lam * w) ** 2)
        assert abs(tau_from_B(Bs[n], prm)[1] - ref) < 1e-7


def test_saramito_elastic_solid_limit():
    """Large Bi (Fig. uncoupl b, Bi = 300): the material never yields and responds
    as a neo-Hookean solid, tau_xy = (mu_p/lam) gamma(t), tau_xx = (mu_p/lam) gamma(t)^2."""
    w, g0 = 1.0, 0.05
    prm = Params('saramito', mu_s=0.0, mu_p=1.0, lam=0.1, tau_y=300.0)
    Lf = lambda t: [[0.0, g0 * w * np.cos(w * t), 0.0], [0.0] * 3, [0.0] * 3]
    ts, Bs = integrate_homogeneous(prm, Lf, 4.0, 1e-3)
    G = prm.mu_p / prm.lam
    for n in (700, 2500, 4000):
        gam = g0 * np.sin(w * ts[n])
        tau = tau_from_B(Bs[n], prm)
        assert closure(Bs[n], prm)[0] == 0.0
        assert abs(tau[1] - G * gam) < 1e-8
        assert abs(tau[0] - G * gam ** 2) < 1e-8


def test_neo_hookean_shear_is_elastic():
    """Table 1 first row (F = a = 0): homogeneous shear gives the elastic closed
    form B_xy = gdot t, B_xx = 1 + (gdot t)^2, tau = G B with no relaxation."""
    prm = Params.from_groups('neo_hookean', Re=1.0, Wi=2.0, beta=0.4)
    G = prm.mu_p / prm.lam
    ts, Bs = integrate_homogeneous(prm, shear_L(0.8), 3.0, 1e-3)
    for n in (500, 1500, 3000):
        t = ts[n]
        assert abs(Bs[n][1] - 0.8 * t) < 1e-10
        assert abs(Bs[n][0] - (1 + (0.8 * t) ** 2)) < 1e-9
        assert abs(tau_from_B(Bs[n], prm)[1] - G * 0.8 * t) < 1e-10
        assert abs(Bs[n][3] - 1.0) < 1e-14
