"""Low-storage RK3 time step (Sec. 3.3.1, Eqs. RK-rt, NS-num1, rk3tau, rk3, NS-num2,
NS-num3, RK).  TEST INFRASTRUCTURE ONLY.

One step advances (u, p, B) from t^n to t^n + dt in three substeps k = 1, 2, 3:

  B^k  = B^{k-1} + dt (zeta^k RT^{k-1} + xi^k RT^{k-2})                (rk3tau)
  u*   = u^{k-1} + dt [zeta^k N^{k-1} + xi^k N^{k-2} - 2 alpha^k grad p^{k-1}
                       + alpha^k (div tau^k + div tau^{k-1})]          (NS-num1, rk3)
  lap psi^k = div u* / (2 alpha^k dt);  p^k = p^{k-1} + psi^k;
  u^k  = u* - 2 alpha^k dt grad psi^k                                  (NS-num2, NS-num3)

with N = -div(uu) + div[mu_s(grad u + grad u^T)] + f.  Reading 3: the paper writes
the viscous term with weights alpha^k at levels k and k-1, which would need an
implicit solve it never describes; the viscous term is taken explicitly with the
advective weights (zeta^k + xi^k = 2 alpha^k for every k, so the total weight per
substep is unchanged), while div(tau) keeps alpha^k at levels k and k-1 because
B^k is known before u* is formed.  The body force f carries the same weights.

Reading 18 (option ``implicit_viscous``, Eq. NS-num1 read literally, uniform
mu_s): the viscous term keeps alpha^k at levels k-1 (explicit) and k (implicit,
Crank-Nicolson within the substep), N holds -div(uu) + f only, and u* solves
  u* - alpha^k dt mu_s lap(u*) = u^{k-1} + dt [zeta^k N^{k-1} + xi^k N^{k-2}
      - 2 alpha^k grad p^{k-1} + alpha^k (div tau^k + div tau^{k-1}) + alpha^k mu_s lap(u^{k-1})]
per component, with that component's wall rule (``poisson.solve_helmholtz``).

Soft particles (``State.phis``, Sec. 3.3.2, Reading 21; neo-Hookean model only):
the solid volume fraction phi_s is advected like B (WENO5 u.grad phi_s with the
RK3 weights and its own history), B evolves with the neo-Hookean closure (F = a
= 0) everywhere, and the extra stress is tau = phi_s G (B - I), G = mu_p/lambda:
elastic in the solid, zero in the (Newtonian) fluid, zero for B = I.

Rigid particles (``State.particles``, Sec. 3.3.2): after u* (and any implicit
viscous solve or penalisation) the discrete-forcing IBM of ``ibm`` turns u* into
u** before the projection; the centres then advance with their prescribed
velocity over the substep.
"""

from dataclasses import dataclass, field

import numpy as np

from .models import tau_from_B
from .momentum import div_tau, grad_p, laplacian, momentum_rhs_n
from .poisson import project, solve_helmholtz
from . import ibm
from .stress import centre_velocity, stress_rhs
from .weno import weno5_derivative

# Eq. RK
RK3_ALPHA = (4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0)
RK3_ZETA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK3_XI = (0.0, -17.0 / 60.0, -5.0 / 12.0)


@dataclass
class State:
    """Prognostic fields on the staggered grid plus the RK3 history terms."""
    U: np.ndarray
    V: np.ndarray
    W: np.ndarray
    p: np.ndarray
    B: list
    RT_hist: list = field(default=None)
    N_hist: tuple = field(default=None)
    t: float = 0.0
    nstep: int = 0
    psi: np.ndarray = field(default=None)
    particles: list = field(default=None)     # rigid particles of the IBM (Reading 19)
    particle_forces: list = field(default=None)
    phis: np.ndarray = field(default=None)     # solid fraction of soft particles (Reading 21)
    phis_hist: np.ndarray = field(default=None)

    @staticmethod
    def rest(g, U=None, V=None, W=None):
        """Velocity as given (zero if None), p = 0 and B = I (tau = 0)."""
        z = g.zeros
        B = [np.ones(g.shape) if d else np.zeros(g.shape)
             for d in (True, False, False, True, False, True)]
        return State(U=z() if U is None else np.array(U, dtype=float),
                     V=z() if V is None else np.array(V, dtype=float),
                     W=z() if W is None else np.array(W, dtype=float),
                     p=z(), B=B)

    def copy(self):
        cp = lambda a: None if a is None else np.array(a, copy=True)
        cl = lambda l: None if l is None else [np.array(a, copy=True) for a in l]
        parts = None if self.particles is None else [dict(q, centre=tuple(q['centre'])) for q in self.particles]
        return State(cp(self.U), cp(self.V), cp(self.W), cp(self.p), cl(self.B),
                     cl(self.RT_hist), None if self.N_hist is None else tuple(cl(self.N_hist)),
                     self.t, self.nstep, cp(self.psi), parts, self.particle_forces, cp(self.phis),
                     cp(self.phis_hist))


def rk3_substep(s, k, dt, g, prm, force=None, solid=None, implicit_viscous=False, ibm_iters=3, gravity=0.0,
                predictor_only=False):
    """Substep k (0-based index into Eq. RK) of the RK3 scheme; returns a new State.

    ``solid`` (optional triple of face arrays alpha) switches on the volume-penalisation
    IBM for fixed obstacles (Sec. 3.3.2, Eqs. Vol, forceAdded): the predicted
    velocity becomes u** = (1 - alpha) u* before the projection, alpha being the
    solid volume fraction of the control volume around each velocity node.

    ``predictor_only`` stops before the projection and returns (u*, B^k): the
    predicted face velocities (with every option above applied) and the updated
    conformation.  Both are local in the fields of level k-1, unlike the
    projection, which is a global solve."""
    alpha, zeta, xi = RK3_ALPHA[k], RK3_ZETA[k], RK3_XI[k]
    has_stress = prm.model != 'newtonian'
    soft = s.phis is not None
    if soft:
        # Reading 21: phi_s advected like B (WENO5, RK3 weights), tau = phi_s G (B - I)
        assert prm.model == 'neo_hookean'
        uc, vc, wc = centre_velocity(s.U, s.V, s.W, g)
        Rphi = -(uc * weno5_derivative(s.phis, g, 'x', uc) + vc * weno5_derivative(s.phis, g, 'y', vc)
                 + wc * weno5_derivative(s.phis, g, 'z', wc))
        inc = zeta * Rphi + (xi * s.phis_hist if xi != 0.0 else 0.0)
        phis_new = s.phis + dt * inc
        gmod = prm.mu_p / prm.lam
        def soft_tau(B, phi):
            return [phi * gmod * (B[c] - (1.0 if c in (0, 3, 5) else 0.0)) for c in range(6)]
    # stress update, Eq. rk3tau with RT of Eq. RK-rt
    if has_stress:
        RT = stress_rhs(s.U, s.V, s.W, s.B, g, prm)
        Bn = []
        for c in range(6):
            inc = zeta * RT[c]
            if xi != 0.0:
                inc = inc + xi * s.RT_hist[c]
            Bn.append(s.B[c] + dt * inc)
    else:
        RT, Bn = None, [b.copy() for b in s.B]
    # momentum predictor, Eqs. NS-num1 and rk3
    N = momentum_rhs_n(s.U, s.V, s.W, g, 0.0 if implicit_viscous else prm.mu_s, force)
    gp = grad_p(s.p, g)
    if has_stress and soft:
        dto = div_tau(soft_tau(s.B, s.phis), g)
        dtn = div_tau(soft_tau(Bn, phis_new), g)
    elif has_stress:
        dto = div_tau(tau_from_B(s.B, prm), g)
        dtn = div_tau(tau_from_B(Bn, prm), g)
    vel = (s.U, s.V, s.W)
    star = []
    for d in range(3):
        inc = zeta * N[d]
        if xi != 0.0:
            inc = inc + xi * s.N_hist[d]
        inc = inc - 2.0 * alpha * gp[d]
        if has_stress:
            inc = inc + alpha * (dtn[d] + dto[d])
        if implicit_viscous:
            inc = inc + alpha * prm.mu_s * laplacian(vel[d], g, 'v' if d == 1 else 'u')
        star.append(vel[d] + dt * inc)
    if implicit_viscous:
        if g.walls:
            star[1][:, g.ny - 1, :] = 0.0
        c = alpha * dt * prm.mu_s
        star = [solve_helmholtz(star[d], g, c, 'v' if d == 1 else 'u') for d in range(3)]
    if solid is not None:
        star = [(1.0 - solid[d]) * star[d] for d in range(3)]
    pforces = None
    if s.particles:
        # discrete-forcing IBM of rigid particles (Eqs. IBM a-d, CoVe2) over the
        # substep's time increment, particles at their positions of level k-1;
        # inner-fluid integrals of free particles before and after (Reading 20)
        I0 = [ibm.inner_integrals(s.U, s.V, s.W, g, q['centre'], q['radius']) if q.get('rho', 0.0) > 0.0 else None
              for q in s.particles]
        star, pforces = ibm.force(star, g, s.particles, 2.0 * alpha * dt, ibm_iters)
        I1 = [ibm.inner_integrals(star[0], star[1], star[2], g, q['centre'], q['radius'])
              if q.get('rho', 0.0) > 0.0 else None for q in s.particles]
    if g.walls:
        star[1][:, g.ny - 1, :] = 0.0
    if predictor_only:
        return star, Bn
    # projection, Eqs. NS-num2 and NS-num3
    U, V, W, psi = project(star[0], star[1], star[2], g, 2.0 * alpha * dt)
    parts = None
    if s.particles:
        parts = [ibm.particle_update(q, f[0], f[1], a, b, 2.0 * alpha * dt, gravity)
                 for q, f, a, b in zip(s.particles, pforces, I0, I1)]
    return State(U=U, V=V, W=W, p=s.p + psi, B=Bn, RT_hist=RT, N_hist=N,
                 t=s.t + (alpha * 2.0) * dt, nstep=s.nstep, psi=psi, particles=parts, particle_forces=pforces,
                 phis=phis_new if soft else None, phis_hist=Rphi if soft else None)


def rk3_step(s, dt, g, prm, force=None, solid=None, implicit_viscous=False, ibm_iters=3, gravity=0.0):
    """One full RK3 step (three substeps); ``solid``, ``implicit_viscous`` and the
    IBM options as in rk3_substep."""
    for k in range(3):
        s = rk3_substep(s, k, dt, g, prm, force, solid, implicit_viscous, ibm_iters, gravity)
    s.nstep += 1
    return s
