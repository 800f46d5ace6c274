"""Monitoring quantities of a state.  TEST INFRASTRUCTURE ONLY.

The paper follows its flows through histories (centre-line velocity, wall shear
stress, B_xx, the yielded region; Sec. 4) and names the loss of positive
definiteness of B as the breakdown it guards against (Sec. 3.1).  The library
summarises a state by the reductions below; each is written here from its
definition on whole arrays, in FP64.

  kinetic energy    1/2 dx dy dz sum over the stored faces of u^2 + v^2 + w^2 (rho = 1)
  max |div u|       of the discrete divergence of ``poisson.divergence``, over the
                    cells where it is finite
  det B, tr B       of the symmetric 3 x 3 conformation at each cell centre
  yielded cells     Saramito (Table 1): cells with F > 0, i.e. |tau^d| > tau_y, with
                    tau = (mu_p/lambda)(B - I); every cell flows for Oldroyd-B and
                    FENE-P (F > 0), none has a yield surface for Newtonian and
                    neo-Hookean (reported as no yielded cells)
  non-finite cells  cells where u, v, w of the faces with the cell's index or a
                    component of B is NaN or infinite
"""

import numpy as np

from .poisson import divergence


def det3_sym(B):
    """det of the symmetric matrix [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]] by
    cofactor expansion along the first row."""
    xx, xy, xz, yy, yz, zz = B
    return xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz)


def deviatoric_magnitude(B, g_mod):
    """|tau^d| = sqrt(1/2 tau^d_ij tau^d_ij) for tau = g_mod (B - I) (Table 1,
    Saramito row); the off-diagonal components are counted twice."""
    t = [g_mod * (B[c] - (1.0 if c in (0, 3, 5) else 0.0)) for c in range(6)]
    tr = t[0] + t[3] + t[5]
    d = [t[c] - (tr / 3.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    return np.sqrt(0.5 * (d[0] * d[0] + d[3] * d[3] + d[5] * d[5]) + d[1] * d[1] + d[2] * d[2] + d[4] * d[4])


def yielded_mask(B, prm):
    """Cells where F of Table 1 is positive."""
    shape = np.shape(B[0])
    if prm.model in ('oldroyd_b', 'fene_p'):
        return np.ones(shape, dtype=bool)
    if prm.model != 'saramito':
        return np.zeros(shape, dtype=bool)
    if prm.tau_y == 0.0:
        return np.ones(shape, dtype=bool)
    return deviatoric_magnitude(B, prm.mu_p / prm.lam) > prm.tau_y


def diagnostics(U, V, W, B, g, prm):
    """All monitoring quantities of a state as a dict.  ``B`` is the list of six
    conformation components (None for a Newtonian state); ``prm`` an
    ``oracle.models.Params``."""
    ke = 0.5 * g.dx * g.dy * g.dz * (np.sum(U * U) + np.sum(V * V) + np.sum(W * W))
    div = divergence(U, V, W, g)
    bad = ~(np.isfinite(U) & np.isfinite(V) & np.isfinite(W))
    ad = np.abs(div)
    ad = ad[np.isfinite(ad)]
    out = dict(kinetic_energy=float(ke), max_div=float(ad.max()) if ad.size else 0.0)
    if B is None:
        out.update(min_det_B=np.inf, max_tr_B=0.0, max_tr_B_over_L2=0.0, yielded_cells=0)
    else:
        for c in range(6):
            bad |= ~np.isfinite(B[c])
        with np.errstate(invalid='ignore', over='ignore'):
            det = det3_sym(B)
            tr = B[0] + B[3] + B[5]
        out['min_det_B'] = float(np.nanmin(det))
        out['max_tr_B'] = float(np.nanmax(tr))
        out['max_tr_B_over_L2'] = out['max_tr_B'] / prm.L2 if prm.model == 'fene_p' else 0.0
        with np.errstate(invalid='ignore', over='ignore'):
            out['yielded_cells'] = int(np.count_nonzero(yielded_mask(B, prm)))
    out['nonfinite_cells'] = int(np.count_nonzero(bad))
    out['yielded_fraction'] = out['yielded_cells'] / g.ncells
    return out
