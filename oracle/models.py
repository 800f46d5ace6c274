"""Constitutive closures of Eq. SRM2 (Sec. 2, Table 1).  TEST INFRASTRUCTURE ONLY.

The generic transport equation for the conformation-like tensor B,

    dB/dt + u.grad B - B.grad u - grad u^T.B = (a/lambda) I - (F/lambda) B,

covers Oldroyd-B, FENE-P and the Saramito elastoviscoplastic model through the
triple (B, F, a) of Table 1.  B is stored as six components in the order
(xx, xy, xz, yy, yz, zz).

Reading 1 (scalings): rho = 1, mu_s = beta/Re, mu_p = (1-beta)/Re, lambda = Wi,
and the yield stress tau_y = Bi/Re (Bi measured against the viscous stress
mu_0 U/L, Sec. 4.1.3) or tau_y = Bi (Bi measured against rho g L, the drop
definition of Sec. 4.2.3).
Reading 2 (gradient convention): (grad u)_ij = du_j/dx_i, so
B.grad u + grad u^T.B = L B + B L^T with L_ij = du_i/dx_j (upper-convected).
Reading 7: the Saramito factor is max(0, 1 - tau_y/|tau^d|), with F = 0 at
|tau^d| = 0 when tau_y > 0 and F = 1 when tau_y = 0 (Bi = 0 is Oldroyd-B).
Reading 16 (local artificial diffusion, Sec. 3.1): a constant diffusivity
art_diff (the paper says the amount is tuned per case and gives none; 0 = off).
Neo-Hookean (Table 1, first row): B = tau/G with F = a = 0, i.e. no relaxation;
the shear modulus is G = mu_p/lambda (the infinite-relaxation-time limit of a
viscoelastic fluid at fixed modulus, as the paper describes it).
"""

from dataclasses import dataclass

import numpy as np

COMPS = ('xx', 'xy', 'xz', 'yy', 'yz', 'zz')
# (row, col) of each stored component
COMP_IJ = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
DIAG = (True, False, False, True, False, True)

MODELS = ('newtonian', 'oldroyd_b', 'fene_p', 'saramito', 'neo_hookean')


def comp_index(a, b):
    """Storage index of the symmetric component (a, b)."""
    a, b = min(a, b), max(a, b)
    return COMP_IJ.index((a, b))


@dataclass
class Params:
    """Physical coefficients of Eqs. NS and SRM2 (floats, or arrays for a mixture)."""
    model: str
    mu_s: object
    mu_p: object
    lam: object
    tau_y: object = 0.0
    L2: float = 0.0
    art_diff: float = 0.0

    @staticmethod
    def from_groups(model, Re, Wi, beta, Bi=0.0, L2=0.0, bi_def=0, art_diff=0.0):
        """Reading 1: dimensionless groups -> coefficients (rho = 1)."""
        assert model in MODELS
        mu0 = 1.0 / Re
        tau_y = Bi * mu0 if bi_def == 0 else Bi
        return Params(model, beta * mu0, (1.0 - beta) * mu0, Wi, tau_y, L2, art_diff)


def closure(B, prm):
    """(F, a) of Table 1 at every cell."""
    if prm.model in ('oldroyd_b', 'newtonian'):
        return 1.0, 1.0
    if prm.model == 'neo_hookean':
        return 0.0, 0.0
    if prm.model == 'fene_p':
        trB = B[0] + B[3] + B[5]
        F = prm.L2 / (prm.L2 - trB)
        a = prm.L2 / (prm.L2 - 3.0)
        return F, a
    if prm.model == 'saramito':
        # tau = (mu_p / lambda)(B - I), Table 1 row "Saramito"
        g = prm.mu_p / prm.lam
        t = [g * (B[c] - (1.0 if DIAG[c] else 0.0)) for c in range(6)]
        tr = t[0] + t[3] + t[5]
        d = [t[c] - (tr / 3.0 if DIAG[c] else 0.0) for c in range(6)]
        # |tau^d| = sqrt(1/2 tau^d_ij tau^d_ij), off-diagonals counted twice
        mag = np.sqrt(0.5 * (d[0] ** 2 + d[3] ** 2 + d[5] ** 2)
                      + d[1] ** 2 + d[2] ** 2 + d[4] ** 2)
        tau_y = np.broadcast_to(np.asarray(prm.tau_y, dtype=float), np.shape(mag))
        safe = np.where(mag > 0.0, mag, 1.0)
        F = np.where(mag > 0.0, np.maximum(0.0, 1.0 - tau_y / safe),
                     np.where(tau_y > 0.0, 0.0, 1.0))
        return F, F
    raise ValueError(prm.model)


def tau_from_B(B, prm):
    """Extra stress tau from B by inverting the B column of Table 1."""
    g = prm.mu_p / prm.lam
    if prm.model == 'newtonian':
        return [np.zeros_like(B[0]) for _ in range(6)]
    if prm.model == 'fene_p':
        F, a = closure(B, prm)
        return [g * (F * B[c] - (a if DIAG[c] else 0.0)) for c in range(6)]
    if prm.model == 'neo_hookean':
        return [g * B[c] for c in range(6)]
    return [g * (B[c] - (1.0 if DIAG[c] else 0.0)) for c in range(6)]


def ucd_terms(B, L):
    """B.grad u + grad u^T.B = L B + B L^T (Reading 2), six components.

    ``L[i][j]`` = du_i/dx_j; written out component by component."""
    out = []
    for (a, b) in COMP_IJ:
        s = 0.0
        for c in range(3):
            s = s + L[a][c] * B[comp_index(c, b)] + B[comp_index(a, c)] * L[b][c]
        out.append(s)
    return out


def rt_local(B, L, prm):
    """Right-hand side of Eq. SRM2 without the advection term:
    (a I - F B)/lambda + B.grad u + grad u^T.B."""
    F, a = closure(B, prm)
    ucd = ucd_terms(B, L)
    return [((a if DIAG[c] else 0.0) - F * B[c]) / prm.lam + ucd[c] for c in range(6)]
