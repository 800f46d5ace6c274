"""Adams-Bashforth two-phase step (Sec. 3.2.2, Eqs. ab2tau, ab2, rt, ru, var-poisson,
projection) with the level set of Sec. 3.2.1.  TEST INFRASTRUCTURE ONLY.

From t^n to t^n + dt:
  1. advance the level set (TVD-RK3 + WENO5, velocity u^n); every
     ``reinit_every`` steps re-distance it (Eq. reinit); with ``mass_iters`` > 0
     shift it to keep the drop volume of the first step (Reading 17);
  2. mixture properties from H(phi^{n+1}): mu_s, mu_p = X1 H + X2 (1 - H),
     lambda and rho uniform (rho = 1: Boussinesq);
  3. B^{n+1} = B^n + dt (3/2 RT^n - 1/2 RT^{n-1})                    (Eq. ab2tau)
  4. u*      = u^n + dt (3/2 RU^n - 1/2 RU^{n-1})                    (Eq. ab2)
     RU^n = -div(uu)^n + div[mu_s^{n+1}(grad u^n + grad u^n^T)] + div tau^n + f^{n+1}
  5. lap p^{n+1} = div u*/dt;  u^{n+1} = u* - dt grad p^{n+1}        (Eqs. var-poisson, projection)

Reading 11:
  * fluid 1 (phi > 0) is the outer EVP fluid (mu_s = beta/Re, mu_p = (1-beta)/Re);
    fluid 2 (the drop) is Newtonian with total viscosity mu_ratio/Re;
  * tau^n is formed from B^n with mu_p^{n+1} (the properties are updated first);
  * the first step is forward Euler (weights 1, 0); the paper is silent on it;
  * f = CSF force (Eq. fLS) + mean-free Boussinesq buoyancy, see ``levelset``.

With a density contrast (``rho_ratio`` = rho_2/rho_1, rho_1 = 1) the step follows
the constant-coefficient splitting of Eqs. poisson-LS and projection-LS
(Dong-Shen): with p_hat = 2 p^n - p^{n-1} and rho_0 = min(rho_1, rho_2),
  lap p^{n+1} = div[(1 - rho_0/rho) grad p_hat] + (rho_0/dt) div u*,
  u^{n+1} = u* - dt [grad p^{n+1}/rho_0 + (1/rho - 1/rho_0) grad p_hat],
and RU carries 1/rho on the viscous, polymer and surface-tension terms (Eq. ru).
Reading 15: rho at a face is the mean of its two neighbouring centres; gravity g
(along -y) acts through (1 - rho_bar/rho) g per unit mass, rho_bar the domain mean,
since a periodic pressure cannot carry the mean weight; p^{-1} = p^0.
"""

from dataclasses import dataclass

import numpy as np

from . import levelset as ls
from .models import Params, tau_from_B
from .grid import at
from .momentum import advection, div_tau, grad_p, viscous
from .poisson import divergence, project, solve_poisson
from .step import State
from .stress import stress_rhs


@dataclass
class TwoPhase:
    """Coefficients of the two-phase (drop) problem."""
    model: str
    Re: float
    Wi: float
    beta: float
    tau_y: float
    mu_ratio: float = 1.0
    L2: float = 0.0
    eps_cells: float = 1.5
    sigma: float = 0.1
    drho_g: float = 1.0
    reinit_every: int = 10
    reinit_iters: int = 3
    rho_ratio: float = None
    gravity: float = 1.0
    art_diff: float = 0.0
    mass_iters: int = 0

    def mixture(self, H):
        mu_s = self.beta / self.Re * H + self.mu_ratio / self.Re * (1.0 - H)
        mu_p = (1.0 - self.beta) / self.Re * H
        return mu_s, mu_p


def face_mean(c, g):
    """Centre field averaged onto the u, v and w faces."""
    return (0.5 * (c + at(c, g, 'c', i=1)), 0.5 * (c + at(c, g, 'c', j=1)), 0.5 * (c + at(c, g, 'c', k=1)))


def split_projection(star, p_n, p_nm1, rho, dt, g, rho0):
    """Dong-Shen constant-coefficient projection (Eqs. poisson-LS, projection-LS).
    Returns (U, V, W, p^{n+1})."""
    rf = face_mean(rho, g)
    ph = 2.0 * p_n - p_nm1
    gph = grad_p(ph, g)
    flux = [(1.0 - rho0 / rf[d]) * gph[d] for d in range(3)]
    if g.walls:
        flux[1][:, g.ny - 1, :] = 0.0
    r = divergence(*flux, g) + rho0 / dt * divergence(*star, g)
    p_new = solve_poisson(r, g)
    gp = grad_p(p_new, g)
    out = [star[d] - dt * (gp[d] / rho0 + (1.0 / rf[d] - 1.0 / rho0) * gph[d]) for d in range(3)]
    if g.walls:
        out[1][:, g.ny - 1, :] = 0.0
    return out[0], out[1], out[2], p_new


def ab2_levelset(phi, s, dt, g, tp, nstep):
    """Step 1: phi^{n+1} from phi^n and u^n (TVD-RK3 + WENO5 advection, re-distancing
    every ``reinit_every`` steps, the mass-preserving shift of Reading 17)."""
    eps = tp.eps_cells * g.dx
    if tp.mass_iters > 0 and nstep == 0:
        tp.v0 = ls.drop_volume(phi, g, eps)
    phi = ls.advect(phi, s.U, s.V, s.W, g, dt)
    if tp.reinit_every > 0 and (nstep + 1) % tp.reinit_every == 0:
        phi = ls.reinitialise(phi, g, tp.reinit_iters)
    if tp.mass_iters > 0:
        phi = ls.mass_correct(phi, g, eps, tp.v0, tp.mass_iters)
    return phi


def ab2_predictor(s, phi, dt, g, tp, nstep, b_mean=None):
    """Steps 2-4 with ``phi`` = phi^{n+1}.  Returns (u*, B^{n+1}, RT^n, RU^n, rho),
    rho being the centre density with a density contrast and None without one.
    Everything here is local in (u^n, B^n, phi^{n+1}) and the histories, except the
    domain mean that makes the Boussinesq buoyancy mean-free (``b_mean``, see
    ``levelset.interface_force_centres``)."""
    eps = tp.eps_cells * g.dx
    # 2. mixture properties at n+1
    H = ls.heaviside(phi, eps)
    mu_s, mu_p = tp.mixture(H)
    prm = Params(tp.model, mu_s=mu_s, mu_p=mu_p, lam=tp.Wi, tau_y=tp.tau_y, L2=tp.L2, art_diff=tp.art_diff)
    w1, w0 = (1.0, 0.0) if nstep == 0 else (1.5, -0.5)
    # 3. stress, Eq. ab2tau
    RT = stress_rhs(s.U, s.V, s.W, s.B, g, prm)
    Bn = [s.B[c] + dt * (w1 * RT[c] + (w0 * s.RT_hist[c] if w0 else 0.0)) for c in range(6)]
    # 4. momentum, Eq. ab2 with RU of Eq. ru
    A = advection(s.U, s.V, s.W, g)
    Vv = viscous(s.U, s.V, s.W, g, mu_s)
    dtau = div_tau(tau_from_B(s.B, prm), g)
    dens = tp.rho_ratio is not None
    fc = ls.interface_force_centres(phi, g, tp.sigma, eps, 0.0 if dens else tp.drho_g, b_mean)
    F = ls.centres_to_faces(fc, g)
    rho = None
    if dens:
        rho = H + tp.rho_ratio * (1.0 - H)
        rf = face_mean(rho, g)
        rbar = rho.mean()
        grav = (0.0, -tp.gravity, 0.0)
        RU = [-A[d] + (Vv[d] + dtau[d] + F[d]) / rf[d] + (1.0 - rbar / rf[d]) * grav[d] for d in range(3)]
    else:
        RU = [-A[d] + Vv[d] + dtau[d] + F[d] for d in range(3)]
    vel = (s.U, s.V, s.W)
    star = [vel[d] + dt * (w1 * RU[d] + (w0 * s.N_hist[d] if w0 else 0.0)) for d in range(3)]
    if g.walls:
        star[1][:, g.ny - 1, :] = 0.0
    return star, Bn, RT, RU, rho


def ab2_step(s, phi, dt, g, tp, nstep):
    """One AB2 step; ``nstep`` counts completed steps (0 for the first).
    ``s.RT_hist`` / ``s.N_hist`` carry RT^{n-1} / RU^{n-1}.  Returns (State, phi)."""
    phi = ab2_levelset(phi, s, dt, g, tp, nstep)
    star, Bn, RT, RU, rho = ab2_predictor(s, phi, dt, g, tp, nstep)
    # 5. projection with dt
    if rho is not None:
        p_nm1 = s.p if s.psi is None or nstep == 0 else s.psi
        U, V, W, p_new = split_projection(star, s.p, p_nm1, rho, dt, g, min(1.0, tp.rho_ratio))
        # psi carries p^{n} to the next step as its p^{n-1}
        return State(U=U, V=V, W=W, p=p_new, B=Bn, RT_hist=RT, N_hist=RU, t=s.t + dt, nstep=nstep + 1,
                     psi=s.p), phi
    U, V, W, psi = project(star[0], star[1], star[2], g, dt)
    return State(U=U, V=V, W=W, p=psi, B=Bn, RT_hist=RT, N_hist=RU, t=s.t + dt, nstep=nstep + 1, psi=psi), phi
