"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the time step itself.  It samples initial
fields on the staggered grid (face velocities, centred level set) and builds
exactly (discretely) divergence-free random velocities as the discrete curl of a
random vector potential, which is how the workloads in the paper's validation
cases are reproduced synthetically:

  * Taylor-Green velocity (single-phase Oldroyd-B box, 32^3);
  * laminar Poiseuille profile plus a random solenoidal perturbation vanishing
    at the walls (Saramito channel);
  * random solenoidal velocity with a k^-5/3 spectrum (FENE-P turbulence) or a
    flat |k| <= 4 spectrum (serving mix);
  * signed distance to a sphere (level-set drop).

Arrays are float64 numpy arrays of shape (nz, ny, nx), x fastest; a face value
at index i is the one on the +1/2 face of cell i.  Grid geometry is passed as a
small dict: nx, ny, nz, lx, ly, lz, walls_y.
"""

import numpy as np


def geometry(nx, ny, nz, lx, ly, lz, walls_y=False):
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), lx=float(lx), ly=float(ly),
                lz=float(lz), walls_y=bool(walls_y))


def _axes(geo):
    nx, ny, nz = geo['nx'], geo['ny'], geo['nz']
    dx, dy, dz = geo['lx'] / nx, geo['ly'] / ny, geo['lz'] / nz
    y0 = -0.5 * geo['ly'] if geo['walls_y'] else 0.0
    return nx, ny, nz, dx, dy, dz, y0


def taylor_green(geo):
    """u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 sampled at the faces."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    xc = (np.arange(nx) + 0.5) * dx
    xf = (np.arange(nx) + 1.0) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    yf = y0 + (np.arange(ny) + 1.0) * dy
    zc = (np.arange(nz) + 0.5) * dz
    U = np.sin(xf)[None, None, :] * np.cos(yc)[None, :, None] * np.cos(zc)[:, None, None]
    V = -np.cos(xc)[None, None, :] * np.sin(yf)[None, :, None] * np.cos(zc)[:, None, None]
    W = np.zeros((nz, ny, nx))
    return U, V, W


def poiseuille(geo, umax=1.0):
    """Laminar profile u = umax (1 - (2y/ly)^2) at the u faces of a channel."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    yc = y0 + (np.arange(ny) + 0.5) * dy
    eta = 2.0 * yc / geo['ly']
    U = np.broadcast_to((umax * (1.0 - eta ** 2))[None, :, None], (nz, ny, nx)).copy()
    return U, np.zeros_like(U), np.zeros_like(U)


def _curl(Ax, Ay, Az, geo):
    """Discrete curl on the staggered grid.

    Ax lives at (x_i, y_{j+1/2}, z_{k+1/2}), Ay at (x_{i+1/2}, y_j, z_{k+1/2}),
    Az at (x_{i+1/2}, y_{j+1/2}, z_k); Ax and Az carry one extra leading y-row
    (the edge below j = 0) so that y differences need no wrap at walls."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    U = (Az[:, 1:, :] - Az[:, :-1, :]) / dy - (Ay - np.roll(Ay, 1, axis=0)) / dz
    V = ((Ax[:, 1:, :] - np.roll(Ax[:, 1:, :], 1, axis=0)) / dz
         - (Az[:, 1:, :] - np.roll(Az[:, 1:, :], 1, axis=2)) / dx)
    W = (Ay - np.roll(Ay, 1, axis=2)) / dx - (Ax[:, 1:, :] - Ax[:, :-1, :]) / dy
    return U, V, W


def _spectral_potential_periodic(geo, rng, kmin, kmax, amp_of_k, xo, yo, zo):
    """Random real field on a triply periodic box sampled at x = (i + xo) dx,
    y = (j + yo) dy, z = (k + zo) dz: Fourier modes kmin <= |k| <= kmax with
    amplitude amp_of_k(|k|) and random complex coefficients, one inverse 3-D FFT."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    kx = np.fft.fftfreq(nx, 1.0 / nx)[None, None, :]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    mag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    mask = (mag >= kmin) & (mag <= kmax)
    amp = np.where(mask, amp_of_k(np.where(mask, mag, 1.0)), 0.0)
    coef = amp * (rng.standard_normal(mag.shape) + 1j * rng.standard_normal(mag.shape))
    shift = np.exp(2j * np.pi * (kx * xo / nx + ky * yo / ny + kz * zo / nz))
    return np.real(np.fft.ifftn(coef * shift)) * (nx * ny * nz)


def _spectral_potential(geo, rng, kmin, kmax, amp_of_k, y_positions, xo, zo):
    """Random real field periodic in x and z (and y unless walls) sampled on the
    lattice x = (i + xo) dx, z = (k + zo) dz and the y values ``y_positions``."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    kz = np.fft.fftfreq(nz, 1.0 / nz)
    if geo['walls_y']:
        ky = np.arange(0, int(kmax) + 1)          # cosine modes across the channel
    else:
        ky = np.fft.fftfreq(ny, 1.0 / ny)
    out = np.zeros((nz, len(y_positions), nx))
    # half-cell lattice offsets as phase factors, so that one inverse FFT
    # evaluates the plane waves exactly at x = (i + xo) dx, z = (k + zo) dz
    shift = (np.exp(2j * np.pi * kz * zo / nz)[:, None]
             * np.exp(2j * np.pi * kx * xo / nx)[None, :])
    for my in ky:
        mag = np.sqrt(kx[None, :] ** 2 + kz[:, None] ** 2 + my ** 2)
        mask = (mag >= kmin) & (mag <= kmax)
        if not mask.any():
            continue
        amp = np.where(mask, amp_of_k(np.where(mask, mag, 1.0)), 0.0)
        coef = amp * (rng.standard_normal(mag.shape) + 1j * rng.standard_normal(mag.shape))
        plane = np.real(np.fft.ifft2(coef * shift)) * (nx * nz)       # (nz, nx)
        if geo['walls_y']:
            yprof = np.cos(np.pi * my * (y_positions - y0) / geo['ly'])
        else:
            phase = rng.uniform(0.0, 2.0 * np.pi)
            yprof = np.cos(2.0 * np.pi * my * y_positions / geo['ly'] + phase)
        out += plane[:, None, :] * yprof[None, :, None]
    return out


def random_solenoidal(geo, seed, kmax, kmin=1.0, spectrum='flat', wall_envelope=True, periodic_fft=False):
    """Discretely divergence-free random velocity (discrete curl of a random vector
    potential).  ``spectrum`` 'flat' weights all modes 1 <= |k| <= kmax equally,
    'k-5/3' shapes the velocity spectrum like k^-5/3.  With walls the potential is
    multiplied by (1 - (2y/ly)^2)^2 so that v vanishes on both walls.
    ``periodic_fft`` draws a triply periodic potential with one 3-D FFT per
    component (fast on large boxes; a different realisation for the same seed).
    Returned unscaled (the caller normalises)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    if spectrum == 'flat':
        amp = lambda k: 1.0 / k
    elif spectrum == 'k-5/3':
        # |u_k| ~ k |A_k| and E(k) ~ k^2 |u_k|^2 ~ k^-5/3  =>  |A_k| ~ k^(-11/6 - 1)
        amp = lambda k: k ** (-11.0 / 6.0 - 1.0)
    else:
        raise ValueError(spectrum)
    if not geo['walls_y'] and periodic_fft:
        # triply periodic: potentials on their staggered lattices from 3-D FFTs;
        # the extra leading y-row is the periodic image of the last one
        Ax = _spectral_potential_periodic(geo, rng, kmin, kmax, amp, 0.5, 1.0, 1.0)
        Ay = _spectral_potential_periodic(geo, rng, kmin, kmax, amp, 1.0, 0.5, 1.0)
        Az = _spectral_potential_periodic(geo, rng, kmin, kmax, amp, 1.0, 1.0, 0.5)
        Ax = np.concatenate([Ax[:, -1:, :], Ax], axis=1)
        Az = np.concatenate([Az[:, -1:, :], Az], axis=1)
        return _curl(Ax, Ay, Az, geo)
    y_cell = y0 + (np.arange(ny) + 0.5) * dy
    y_edge = y0 + np.arange(-1, ny) * dy + dy        # edges j-1/2 for j = 0..ny
    Ax = _spectral_potential(geo, rng, kmin, kmax, amp, y_edge, 0.5, 1.0)
    Ay = _spectral_potential(geo, rng, kmin, kmax, amp, y_cell, 1.0, 1.0)
    Az = _spectral_potential(geo, rng, kmin, kmax, amp, y_edge, 1.0, 0.5)
    if geo['walls_y'] and wall_envelope:
        env = lambda y: (1.0 - (2.0 * y / geo['ly']) ** 2) ** 2
        Ax *= env(y_edge)[None, :, None]
        Az *= env(y_edge)[None, :, None]
        Ay *= env(y_cell)[None, :, None]
    return _curl(Ax, Ay, Az, geo)


def scale_max(U, V, W, target):
    m = max(np.abs(U).max(), np.abs(V).max(), np.abs(W).max())
    s = target / m if m > 0 else 0.0
    return U * s, V * s, W * s


def scale_rms(U, V, W, target):
    rms = np.sqrt((U ** 2 + V ** 2 + W ** 2).mean() / 3.0)
    s = target / rms if rms > 0 else 0.0
    return U * s, V * s, W * s


def sphere_distance(geo, centre, radius):
    """Signed distance |x - c| - R at cell centres (positive outside the drop)."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    x = (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dy
    z = (np.arange(nz) + 0.5) * dz
    r = np.sqrt((x[None, None, :] - centre[0]) ** 2 + (y[None, :, None] - centre[1]) ** 2
                + (z[:, None, None] - centre[2]) ** 2)
    return r - radius


def random_conformation(geo, seed, amp=0.2):
    """A smooth symmetric positive-definite B field near the identity, for tests:
    B = I + amp * S with S a random smooth symmetric field of max-norm <= 1."""
    rng = np.random.default_rng(seed)
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    x = (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dy
    z = (np.arange(nz) + 0.5) * dz
    B = []
    for c, diag in enumerate((True, False, False, True, False, True)):
        f = np.zeros((nz, ny, nx))
        for _ in range(3):
            mx, my, mz = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            f += (np.sin(2 * np.pi * mx * x / geo['lx'] + ph[0])[None, None, :]
                  * np.cos(2 * np.pi * my * y / geo['ly'] + ph[1])[None, :, None]
                  * np.sin(2 * np.pi * mz * z / geo['lz'] + ph[2])[:, None, None])
        f /= 3.0
        B.append((1.0 if diag else 0.0) + amp * (0.5 if not diag else 1.0) * f)
    return B


def spd_conformation(geo, seed, amp=0.5, scale=1.0):
    """A smooth symmetric positive-definite B field with large deviations, for tests:
    B = scale * M M with M = I + amp * S (S as in ``random_conformation``), components
    in the order xx, xy, xz, yy, yz, zz.  B is positive definite wherever M is
    nonsingular; ``scale`` multiplies its deviatoric part (and its determinant by
    scale^3)."""
    S = random_conformation(geo, seed, amp=1.0)
    m = [S[c] - (1.0 if c in (0, 3, 5) else 0.0) for c in range(6)]
    m = [(1.0 if c in (0, 3, 5) else 0.0) + amp * m[c] for c in range(6)]
    m0, m1, m2, m3, m4, m5 = m
    return [scale * (m0 * m0 + m1 * m1 + m2 * m2),
            scale * (m0 * m1 + m1 * m3 + m2 * m4),
            scale * (m0 * m2 + m1 * m4 + m2 * m5),
            scale * (m1 * m1 + m3 * m3 + m4 * m4),
            scale * (m1 * m2 + m3 * m4 + m4 * m5),
            scale * (m2 * m2 + m4 * m4 + m5 * m5)]


def solid_fractions(geo, inside, samples=4):
    """Solid volume fraction of the control volume around every u, v and w node
    (the cell shifted by half a cell along that component's axis), by sub-sampling
    each control volume on a samples^3 lattice.  ``inside(x, y, z)`` is a
    vectorised predicate of the solid region.  Returns (ax, ay, az)."""
    nx, ny, nz, dx, dy, dz, y0 = _axes(geo)
    off = (np.arange(samples) + 0.5) / samples - 0.5          # sub-cell offsets in cell units
    out = []
    for shift in ((1.0, 0.5, 0.5), (0.5, 1.0, 0.5), (0.5, 0.5, 1.0)):
        # node positions: face of component d, centres in the other two directions
        xs = (np.arange(nx) + shift[0]) * dx
        ys = y0 + (np.arange(ny) + shift[1]) * dy
        zs = (np.arange(nz) + shift[2]) * dz
        acc = np.zeros((nz, ny, nx))
        for ox in off:
            for oy in off:
                for oz in off:
                    X = (xs + ox * dx)[None, None, :]
                    Y = (ys + oy * dy)[None, :, None]
                    Z = (zs + oz * dz)[:, None, None]
                    acc += inside(X + 0 * Y + 0 * Z, Y + 0 * X + 0 * Z, Z + 0 * X + 0 * Y)
        out.append(acc / samples ** 3)
    return tuple(out)
