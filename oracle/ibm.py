"""Discrete-forcing immersed boundary method for rigid particles (Sec. 3.3.2,
Eqs. IBM a-d and CoVe2).  TEST INFRASTRUCTURE ONLY.

Within an RK3 substep, after the predicted velocity u* is formed:
  U*_l   = sum_ijk u*_ijk delta(x_ijk - X_l) dV                  (IBM a, interpolation)
  F_l    = (U(X_l) - U*_l) / dt_s                                 (IBM b)
  f_ijk  = sum_l F_l delta(x_ijk - X_l) dV_l                      (IBM c, spreading)
  u**    = u* + dt_s f                                            (IBM d)
repeated ``iters`` times with u** in place of u* and the Lagrangian forces
accumulated (multi-direct forcing, Eq. CoVe2).  rho_f = 1.

Reading 19 (the paper gives the scheme but not these details):
  * delta is the three-point kernel of Roma et al.:
      phi(r) = (1 + sqrt(1 - 3 r^2)) / 3                     for |r| <= 1/2,
      phi(r) = (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6       for 1/2 <= |r| <= 3/2,
    delta(x) = phi(dx_/dx) phi(dy_/dy) phi(dz_/dz) / (dx dy dz), applied to each
    velocity component on its own staggered lattice;
  * spheres only; the Lagrangian points sit on a sphere retracted by 0.3 dx into
    the particle, R_r = R - 0.3 dx, their number is N_L = round(pi/3 (12 (R_r/dx)^2 + 1))
    and each carries dV_l = pi dx (12 R_r^2 + dx^2)/(3 N_L) (a shell one cell
    thick shared equally); they are spread uniformly by the generalised spiral
    z_l = 1 - (2l + 1)/N_L, azimuth l times the golden angle;
  * the surface velocity is U_p + omega_p x r for a prescribed motion (constant
    U_p, omega_p; the centre moves with U_p); dt_s is the substep's time increment
    2 alpha^k dt (it cancels in u**, only the reported forces depend on it);
  * particles stay at least R + 2 dx away from walls (no wall stencils).
Reading 20 (free motion; the paper gives Eqs. NewtonEulerWim1/2 and says they are
integrated with the RK3 scheme): per substep, with dt_s = 2 alpha^k dt, the
particle's inner-fluid integrals I_u = int_Vp u dV and I_r = int_Vp r x u dV taken
as sums over velocity nodes of phi_s u dV (phi_s = solid fraction of the node's
control volume from 4^3 sub-samples, r from the centre to the node) of u^{k-1}
(before) and of u** (after the forcing), at the centre X^{k-1}:
  rho_p V_p (U^k - U^{k-1}) = -dt_s sum F_l dV_l + (I_u^k - I_u^{k-1}) + dt_s (rho_p - 1) V_p g,
  I_p (omega^k - omega^{k-1}) = -dt_s sum r_l x F_l dV_l + (I_r^k - I_r^{k-1}),
  X^k = X^{k-1} + dt_s (U^k + U^{k-1}) / 2,
rho_f = 1, V_p = 4 pi R^3/3, I_p = 2 rho_p V_p R^2 / 5, g along -y; no collisions.
A prescribed particle keeps U_p and omega_p and moves by dt_s U_p.
"""

import numpy as np

GOLDEN = np.pi * (3.0 - np.sqrt(5.0))


def roma_phi(r):
    """Three-point regularised delta kernel of Roma et al. (one direction, r in cells)."""
    a = np.abs(np.asarray(r, dtype=float))
    out = np.zeros_like(a)
    inner = a <= 0.5
    outer = (a > 0.5) & (a <= 1.5)
    out[inner] = (1.0 + np.sqrt(1.0 - 3.0 * a[inner] ** 2)) / 3.0
    out[outer] = (5.0 - 3.0 * a[outer] - np.sqrt(np.maximum(0.0, 1.0 - 3.0 * (1.0 - a[outer]) ** 2))) / 6.0
    return out


def lagrangian_points(centre, radius, dx):
    """Points (N_L, 3) on the retracted sphere, their offsets r from the centre and dV_l."""
    rr = radius - 0.3 * dx
    n = int(round(np.pi / 3.0 * (12.0 * (rr / dx) ** 2 + 1.0)))
    l = np.arange(n)
    z = 1.0 - (2.0 * l + 1.0) / n
    rho = np.sqrt(1.0 - z * z)
    th = GOLDEN * l
    off = rr * np.stack([rho * np.cos(th), rho * np.sin(th), z], axis=1)
    dvl = np.pi * dx * (12.0 * rr * rr + dx * dx) / (3.0 * n)
    return np.asarray(centre, dtype=float)[None, :] + off, off, dvl


def _lattice(g, comp):
    """Coordinates of component comp's nodes along x, y, z (u: x-faces; v: y-faces; w: z-faces)."""
    y0 = -0.5 * g.ly if g.walls else 0.0
    xc = (np.arange(g.nx) + 0.5) * g.dx
    yc = y0 + (np.arange(g.ny) + 0.5) * g.dy
    zc = (np.arange(g.nz) + 0.5) * g.dz
    xf, yf, zf = xc + 0.5 * g.dx, yc + 0.5 * g.dy, zc + 0.5 * g.dz
    return (xf if comp == 0 else xc), (yf if comp == 1 else yc), (zf if comp == 2 else zc), y0


def _stencil(g, comp, X):
    """Indices (3 per direction) and kernel weights phi of the nodes around point X."""
    xs, ys, zs, y0 = _lattice(g, comp)
    idx, wts = [], []
    for d, (coords, h, n, origin) in enumerate(((xs, g.dx, g.nx, 0.0), (ys, g.dy, g.ny, y0), (zs, g.dz, g.nz, 0.0))):
        # nearest node, then the three around it (periodic index wrap)
        base = int(np.floor((X[d] - coords[0]) / h + 0.5))
        ii = np.array([base - 1, base, base + 1])
        pos = coords[0] + ii * h
        w = roma_phi((pos - X[d]) / h)
        idx.append(ii % n)
        wts.append(w)
    return idx, wts


def interpolate(F, g, comp, pts):
    """U_l = sum over nodes of F delta(x - X_l) dV (Eq. IBM a)."""
    out = np.empty(len(pts))
    for l, X in enumerate(pts):
        (ix, iy, iz), (wx, wy, wz) = _stencil(g, comp, X)
        w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
        out[l] = float((F[np.ix_(iz, iy, ix)] * w).sum())
    return out


def spread(Fl, g, comp, pts, dvl):
    """f = sum_l F_l delta(x - X_l) dV_l on component comp's lattice (Eq. IBM c)."""
    f = np.zeros(g.shape)
    cell = g.dx * g.dy * g.dz
    for l, X in enumerate(pts):
        (ix, iy, iz), (wx, wy, wz) = _stencil(g, comp, X)
        w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
        np.add.at(f, np.ix_(iz, iy, ix), Fl[l] * w * dvl / cell)
    return f


def surface_velocity(p, off):
    """U_p + omega_p x r at the Lagrangian points of particle p (dict with 'u', 'omega')."""
    return np.asarray(p['u'], dtype=float)[None, :] + np.cross(np.asarray(p['omega'], dtype=float)[None, :], off)


def force(star, g, particles, dts, iters):
    """Multi-direct forcing (Eqs. IBM, CoVe2).  Returns (u**, per-particle force and
    torque that the fluid exerts on each particle: -sum_l F_l dV_l and
    -sum_l r_l x F_l dV_l)."""
    ustar = [a.copy() for a in star]
    layout = []
    for p in particles:
        pts, off, dvl = lagrangian_points(p['centre'], p['radius'], g.dx)
        layout.append((pts, off, dvl, surface_velocity(p, off), np.zeros((len(pts), 3))))
    for _ in range(iters):
        # interpolate every point from the current u**, then spread all increments
        incs = []
        for pts, off, dvl, target, Facc in layout:
            dF = np.stack([(target[:, c] - interpolate(ustar[c], g, c, pts)) / dts for c in range(3)], axis=1)
            Facc += dF
            incs.append(dF)
        for (pts, off, dvl, target, Facc), dF in zip(layout, incs):
            for c in range(3):
                ustar[c] = ustar[c] + dts * spread(dF[:, c], g, c, pts, dvl)
    out = []
    for pts, off, dvl, target, Facc in layout:
        out.append((-(Facc * dvl).sum(axis=0), -(np.cross(off, Facc) * dvl).sum(axis=0)))
    return ustar, out


def inner_integrals(U, V, W, g, centre, radius, samples=4):
    """(I_u, I_r): sums of phi_s u dV and phi_s r x u dV over the velocity nodes
    (Reading 20); x and z (and a periodic y) use the minimum-image offset."""
    sub = (np.arange(samples) + 0.5) / samples - 0.5
    cell = g.dx * g.dy * g.dz
    L = (g.lx, g.ly, g.lz)
    periodic = (True, not g.walls, True)
    Iu, Ir = np.zeros(3), np.zeros(3)
    for comp, F in enumerate((U, V, W)):
        xs, ys, zs, y0 = _lattice(g, comp)
        def rel(c, d):
            r = c - centre[d]
            if periodic[d]:
                r = (r + 0.5 * L[d]) % L[d] - 0.5 * L[d]
            return r
        rx = rel(xs, 0)[None, None, :]
        ry = rel(ys, 1)[None, :, None]
        rz = rel(zs, 2)[:, None, None]
        frac = np.zeros(g.shape)
        for ox in sub:
            for oy in sub:
                for oz in sub:
                    d2 = (rx + ox * g.dx) ** 2 + (ry + oy * g.dy) ** 2 + (rz + oz * g.dz) ** 2
                    frac += d2 < radius * radius
        w = frac / samples ** 3 * cell * F
        r = (rx + 0 * w, ry + 0 * w, rz + 0 * w)
        Iu[comp] += w.sum()
        # r x u: with (c, a, b) cyclic, (r x u)_a gains r_b u_c and (r x u)_b loses r_a u_c
        a, b = (comp + 1) % 3, (comp + 2) % 3
        Ir[a] += (r[b] * w).sum()
        Ir[b] -= (r[a] * w).sum()
    return Iu, Ir


def particle_update(p, force, torque, I0, I1, dts, gravity):
    """Reading 20: one substep of the Newton-Euler equations of a free sphere
    (``p['rho']`` > 0) or of a prescribed one; returns the updated particle."""
    c = np.asarray(p['centre'], dtype=float)
    u0 = np.asarray(p['u'], dtype=float)
    if p.get('rho', 0.0) > 0.0:
        R, rho = p['radius'], p['rho']
        vp = 4.0 / 3.0 * np.pi * R ** 3
        ip = 0.4 * rho * vp * R * R
        g = np.array([0.0, -gravity, 0.0])
        u1 = u0 + (dts * np.asarray(force) + (I1[0] - I0[0]) + dts * (rho - 1.0) * vp * g) / (rho * vp)
        w1 = np.asarray(p['omega'], dtype=float) + (dts * np.asarray(torque) + (I1[1] - I0[1])) / ip
        return dict(p, centre=tuple(c + 0.5 * dts * (u1 + u0)), u=tuple(u1), omega=tuple(w1))
    return dict(p, centre=tuple(c + dts * u0))

