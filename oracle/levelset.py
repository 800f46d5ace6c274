"""Level set, interface forces and mixture properties of the two-phase step
(Sec. 3.2.1: Eqs. fLS, ls-adv, normal, curv, reinit and the mixture rule).
TEST INFRASTRUCTURE ONLY.

phi > 0 is fluid 1 (the bulk), phi < 0 fluid 2 (the drop); phi = 0 is the
interface.  Reading 10 (the paper cites Ge et al. for the details it omits):
  * H(phi) = 0 for phi < -eps, 1 for phi > eps, (1 + phi/eps + sin(pi phi/eps)/pi)/2
    in between; delta = dH/dphi; eps = eps_cells * dx;
  * advection u.grad(phi) by the same upwind WENO5 as B (Sec. 3.1), integrated
    with the three-stage TVD Runge-Kutta scheme (Shu-Osher), velocity frozen at u^n;
  * reinitialisation: a few pseudo-time steps (dtau = 0.5 dx) of
    d phi/d tau + S(phi0)(|grad phi| - 1) = 0 with S(phi0) = phi0/sqrt(phi0^2 + dx^2),
    |grad phi| from the Godunov upwind combination of the WENO5 one-sided
    derivatives, TVD-RK3 in pseudo-time;
  * n = grad(phi)/|grad(phi)| and kappa = -div(n), both by central differences at
    cell centres (|grad phi| floored at 1e-12);
  * CSF force sigma kappa delta(phi) n at cell centres (Eq. fLS), averaged onto faces;
  * Boussinesq buoyancy +(1 - H) drho_g along y at centres, minus its domain mean
    (a periodic box has no net acceleration), averaged onto v faces.
Reading 17 (mass conservation; the paper names a mass-conserving interface-
correction level set and cites Ge et al. for it without giving the correction):
after each level-set step phi is shifted uniformly, phi <- phi + d, with d from
Newton iterations on the smoothed volume of fluid 2, V(phi) = sum (1 - H(phi)) dV,
whose derivative is dV/dd = -sum delta(phi) dV, so that V returns to its value
at the first step.
"""

import numpy as np

from .grid import at
from .stress import centre_velocity
from .weno import weno5_derivative, weno5_one_sided


def heaviside(phi, eps):
    inner = 0.5 * (1.0 + phi / eps + np.sin(np.pi * phi / eps) / np.pi)
    return np.where(phi < -eps, 0.0, np.where(phi > eps, 1.0, inner))


def delta(phi, eps):
    inner = 0.5 / eps * (1.0 + np.cos(np.pi * phi / eps))
    return np.where(np.abs(phi) > eps, 0.0, inner)


def advection_rhs(phi, U, V, W, g):
    """-u.grad(phi) with u at the cell centres, WENO5 upwinded (Eq. ls-adv)."""
    uc, vc, wc = centre_velocity(U, V, W, g)
    return -(uc * weno5_derivative(phi, g, 'x', uc) + vc * weno5_derivative(phi, g, 'y', vc)
             + wc * weno5_derivative(phi, g, 'z', wc))


def tvd_rk3(phi, rhs, dt):
    """Three-stage TVD Runge-Kutta (Shu-Osher) for d phi/dt = rhs(phi)."""
    p1 = phi + dt * rhs(phi)
    p2 = 0.75 * phi + 0.25 * (p1 + dt * rhs(p1))
    return phi / 3.0 + 2.0 / 3.0 * (p2 + dt * rhs(p2))


def advect(phi, U, V, W, g, dt):
    return tvd_rk3(phi, lambda f: advection_rhs(f, U, V, W, g), dt)


def godunov_grad_norm(phi, sgn, g):
    """|grad phi| by Godunov's upwind rule from the one-sided WENO5 derivatives:
    for S > 0 each direction contributes max(max(a, 0)^2, min(b, 0)^2), for S <= 0
    max(min(a, 0)^2, max(b, 0)^2), with a the left-biased and b the right-biased
    derivative."""
    tot = 0.0
    for axis in ('x', 'y', 'z'):
        a, b = weno5_one_sided(phi, g, axis)
        pos = np.maximum(np.maximum(a, 0.0) ** 2, np.minimum(b, 0.0) ** 2)
        neg = np.maximum(np.minimum(a, 0.0) ** 2, np.maximum(b, 0.0) ** 2)
        tot = tot + np.where(sgn > 0.0, pos, neg)
    return np.sqrt(tot)


def reinit_rhs(phi, phi0, g):
    """-S(phi0)(|grad phi| - 1) of Eq. reinit."""
    h = g.dx
    sgn = phi0 / np.sqrt(phi0 ** 2 + h ** 2)
    return -sgn * (godunov_grad_norm(phi, sgn, g) - 1.0)


def reinitialise(phi, g, iters, dtau_cells=0.5):
    phi0 = phi.copy()
    dtau = dtau_cells * g.dx
    for _ in range(iters):
        phi = tvd_rk3(phi, lambda f: reinit_rhs(f, phi0, g), dtau)
    return phi


def normals(phi, g):
    """n = grad(phi)/|grad(phi)| by central differences at centres (Eq. normal)."""
    gx = (at(phi, g, 'c', i=1) - at(phi, g, 'c', i=-1)) / (2.0 * g.dx)
    gy = (at(phi, g, 'c', j=1) - at(phi, g, 'c', j=-1)) / (2.0 * g.dy)
    gz = (at(phi, g, 'c', k=1) - at(phi, g, 'c', k=-1)) / (2.0 * g.dz)
    mag = np.maximum(np.sqrt(gx ** 2 + gy ** 2 + gz ** 2), 1e-12)
    return gx / mag, gy / mag, gz / mag


def curvature(n, g):
    """kappa = -div(n) by central differences at centres (Eq. curv)."""
    nx, ny, nz = n
    return -((at(nx, g, 'c', i=1) - at(nx, g, 'c', i=-1)) / (2.0 * g.dx)
             + (at(ny, g, 'c', j=1) - at(ny, g, 'c', j=-1)) / (2.0 * g.dy)
             + (at(nz, g, 'c', k=1) - at(nz, g, 'c', k=-1)) / (2.0 * g.dz))


def interface_force_centres(phi, g, sigma, eps, drho_g, b_mean=None):
    """CSF force sigma kappa delta(phi) n (Eq. fLS) plus the mean-free Boussinesq
    buoyancy (1 - H) drho_g e_y, at cell centres.  ``b_mean`` (default: the mean over
    ``phi``'s cells) is the domain mean of (1 - H) drho_g that makes it mean-free;
    a caller passing a window of a larger field passes the larger field's mean."""
    n = normals(phi, g)
    kap = curvature(n, g)
    dl = delta(phi, eps)
    fx = sigma * kap * dl * n[0]
    fy = sigma * kap * dl * n[1]
    fz = sigma * kap * dl * n[2]
    b = (1.0 - heaviside(phi, eps)) * drho_g
    fy = fy + b - (b.mean() if b_mean is None else b_mean)
    return fx, fy, fz


def centres_to_faces(fc, g):
    """Face values as the mean of the two neighbouring centres."""
    fx, fy, fz = fc
    Fx = 0.5 * (fx + at(fx, g, 'c', i=1))
    Fy = 0.5 * (fy + at(fy, g, 'c', j=1))
    Fz = 0.5 * (fz + at(fz, g, 'c', k=1))
    if g.walls:
        Fy[:, g.ny - 1, :] = 0.0
    return Fx, Fy, Fz


def drop_volume(phi, g, eps):
    """Smoothed volume of fluid 2 (phi < 0): sum of 1 - H(phi) over the cells."""
    return float((1.0 - heaviside(phi, eps)).sum()) * g.dx * g.dy * g.dz


def mass_correct(phi, g, eps, v0, iters):
    """Reading 17: uniform shift of phi restoring the smoothed drop volume v0,
    ``iters`` Newton iterations d <- d + (V(phi + d) - v0) / A(phi + d) with
    A = sum delta(phi + d) dV."""
    dv = g.dx * g.dy * g.dz
    d = 0.0
    for _ in range(iters):
        p = phi + d
        v = float((1.0 - heaviside(p, eps)).sum()) * dv
        a = float(delta(p, eps).sum()) * dv
        if a > 0.0:
            d += (v - v0) / a
    return phi + d

