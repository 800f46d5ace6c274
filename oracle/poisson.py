"""Fast Poisson solver and projection (Eqs. var-poisson, projection, NS-num2, NS-num3).
TEST INFRASTRUCTURE ONLY.

The pressure-like variable psi solves the discrete Poisson equation
lap(psi) = r with the 7-point Laplacian of the staggered grid.  It is solved by
FFTs in the periodic directions (numpy.fft as the library step) and, along a
wall-bounded y, by a tridiagonal (Thomas) solve per Fourier mode (Sec. 3.2.2
"efficient FFT-based pressure solver").

Reading 9: the modal eigenvalues are those of the discrete Laplacian,
lambda(m) = (2 - 2 cos(2 pi m / n)) / h^2, so that the projection is exact; the
periodic zero mode is set to zero; with walls psi has Neumann rows at j = 0 and
j = ny-1 (the missing neighbour and its coefficient dropped), and the singular
(kx, kz) = (0, 0) system is pinned by replacing its first row with psi_0 = 0.
The same transforms solve the Helmholtz problems of the implicit viscous option
(``solve_helmholtz``, Reading 18).
"""

import numpy as np

from .grid import at


def divergence(U, V, W, g):
    """Discrete divergence at cell centres (walls: the face below j = 0 has v = 0)."""
    return ((U - at(U, g, 'u', i=-1)) / g.dx
            + (V - at(V, g, 'v', j=-1)) / g.dy
            + (W - at(W, g, 'u', k=-1)) / g.dz)


def eigenvalues(n, h):
    """lambda(m) = (2 - 2 cos(2 pi m / n)) / h^2 for m = 0..n-1 (numpy FFT order)."""
    m = np.arange(n)
    return (2.0 - 2.0 * np.cos(2.0 * np.pi * m / n)) / h ** 2


def thomas(lower, diag, upper, rhs):
    """Thomas algorithm for tridiagonal systems along axis 0 of ``rhs``.

    ``lower[j]`` multiplies x[j-1], ``diag[j]`` x[j], ``upper[j]`` x[j+1]; the
    coefficient arrays broadcast against ``rhs[j]``.  Forward elimination, then
    back substitution."""
    n = rhs.shape[0]
    cp = [None] * n
    dp = [None] * n
    cp[0] = upper[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for j in range(1, n):
        m = diag[j] - lower[j] * cp[j - 1]
        cp[j] = upper[j] / m
        dp[j] = (rhs[j] - lower[j] * dp[j - 1]) / m
    x = np.empty_like(rhs)
    x[n - 1] = dp[n - 1]
    for j in range(n - 2, -1, -1):
        x[j] = dp[j] - cp[j] * x[j + 1]
    return x


def solve_poisson(r, g):
    """psi with lap(psi) = r (Eq. NS-num2 with its right-hand side given)."""
    lx = eigenvalues(g.nx, g.dx)[None, None, :]
    lz = eigenvalues(g.nz, g.dz)[:, None, None]
    if not g.walls:
        ly = eigenvalues(g.ny, g.dy)[None, :, None]
        rh = np.fft.fftn(r)
        lam = lx + ly + lz
        lam_safe = np.where(lam == 0.0, 1.0, lam)
        ph = np.where(lam == 0.0, 0.0, -rh / lam_safe)
        return np.real(np.fft.ifftn(ph))
    # walls: FFT in x and z, tridiagonal along y per (kz, kx)
    rh = np.fft.fft(np.fft.fft(r, axis=2), axis=0)          # (nz, ny, nx) complex
    ny, idy2 = g.ny, 1.0 / g.dy ** 2
    lam = (lx + lz)[:, 0, :]                               # (nz, nx)
    lower = np.full((ny,) + lam.shape, idy2)
    upper = np.full((ny,) + lam.shape, idy2)
    diag = np.broadcast_to(-2.0 * idy2 - lam, (ny,) + lam.shape).copy()
    # Neumann rows: drop the missing neighbour and its -1/dy^2
    lower[0] = 0.0
    upper[ny - 1] = 0.0
    diag[0] += idy2
    diag[ny - 1] += idy2
    rhs = np.moveaxis(rh, 1, 0).copy()                      # (ny, nz, nx)
    # pin the singular (0, 0) mode with psi_0 = 0
    diag[0, 0, 0] = 1.0
    upper[0, 0, 0] = 0.0
    rhs[0, 0, 0] = 0.0
    ph = thomas(lower, diag, upper, rhs)
    ph = np.moveaxis(ph, 0, 1)
    return np.real(np.fft.ifft(np.fft.ifft(ph, axis=0), axis=2))


def solve_helmholtz(r, g, c, kind):
    """x with x - c lap(x) = r for a velocity component, lap the 7-point Laplacian
    with that component's ghost rule (Reading 18): 'u' (u or w, centred in y; at
    walls the odd no-slip mirror x_{-1} = -x_0, x_ny = -x_{ny-1}) or 'v' (y-faces;
    at walls x = 0 on the bottom wall face below j = 0 and on the stored top face
    j = ny-1, so rows 0 .. ny-2 are solved and row ny-1 is zero)."""
    lx = eigenvalues(g.nx, g.dx)[None, None, :]
    lz = eigenvalues(g.nz, g.dz)[:, None, None]
    if not g.walls:
        ly = eigenvalues(g.ny, g.dy)[None, :, None]
        return np.real(np.fft.ifftn(np.fft.fftn(r) / (1.0 + c * (lx + ly + lz))))
    rh = np.fft.fft(np.fft.fft(r, axis=2), axis=0)
    ny, cy = g.ny, c / g.dy ** 2
    lam = (lx + lz)[:, 0, :]
    m = ny if kind == 'u' else ny - 1                      # unknown rows
    lower = np.full((m,) + lam.shape, -cy)
    upper = np.full((m,) + lam.shape, -cy)
    diag = np.broadcast_to(1.0 + c * lam + 2.0 * cy, (m,) + lam.shape).copy()
    lower[0] = 0.0
    upper[m - 1] = 0.0
    if kind == 'u':
        # odd mirror: the ghost -x_0 (-x_{ny-1}) folds into the diagonal
        diag[0] += cy
        diag[m - 1] += cy
    rhs = np.moveaxis(rh, 1, 0)[:m].copy()
    xh = thomas(lower, diag, upper, rhs)
    out = np.zeros((ny,) + lam.shape, dtype=complex)
    out[:m] = xh
    out = np.moveaxis(out, 0, 1)
    return np.real(np.fft.ifft(np.fft.ifft(out, axis=0), axis=2))


def project(U, V, W, g, coef):
    """One projection: lap(psi) = div(u*)/coef, u = u* - coef grad(psi).

    ``coef`` is 2 alpha^k dt for the RK3 substep (Eqs. NS-num2/3), dt for the AB2
    step (Eqs. var-poisson, projection, rho = 1).  Returns (U, V, W, psi)."""
    r = divergence(U, V, W, g) / coef
    psi = solve_poisson(r, g)
    Un = U - coef * (at(psi, g, 'c', i=1) - psi) / g.dx
    Vn = V - coef * (at(psi, g, 'c', j=1) - psi) / g.dy
    Wn = W - coef * (at(psi, g, 'c', k=1) - psi) / g.dz
    if g.walls:
        Vn[:, g.ny - 1, :] = 0.0
    return Un, Vn, Wn, psi
