"""Pins for the oracle's fast Poisson solver and projection (Eqs. NS-num2, NS-num3)."""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.linalg import solve_banded

import oracle
from oracle.poisson import thomas, eigenvalues
from paper_1803_09563_gb300 import inputs


def grid(nx, ny, nz, walls):
    return oracle.Grid(nx, ny, nz, 2 * np.pi, 2.0 if walls else 2 * np.pi, 2 * np.pi, walls)


def laplacian_matrix(g):
    """7-point Laplacian assembled independently as a sparse matrix (periodic x, z;
    y periodic or Neumann)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    N = nx * ny * nz
    idx = lambda i, j, k: (k * ny + j) * nx + i
    rows, cols, vals = [], [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                for (di, dj, dk, h) in ((1, 0, 0, g.dx), (-1, 0, 0, g.dx), (0, 1, 0, g.dy),
                                        (0, -1, 0, g.dy), (0, 0, 1, g.dz), (0, 0, -1, g.dz)):
                    jj = j + dj
                    if g.walls and (jj < 0 or jj >= ny):
                        continue            # Neumann: no flux through the wall
                    c = idx((i + di) % nx, jj % ny, (k + dk) % nz)
                    rows += [r, r]
                    cols += [c, r]
                    vals += [1.0 / h ** 2, -1.0 / h ** 2]
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


@pytest.mark.parametrize("walls", [False, True])
def test_solution_matches_sparse_direct_solve(walls):
    g = grid(6, 5, 4, walls)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(g.shape)
    r -= r.mean()                    # compatibility: zero net source
    psi = oracle.solve_poisson(r, g)
    A = laplacian_matrix(g)
    # residual of the oracle's psi in the independent operator
    res = A @ psi.ravel() - r.ravel()
    assert np.abs(res).max() < 1e-10
    # and equal, up to the additive constant, to a direct solve with one value pinned
    A2 = A.tolil()
    A2[0, :] = 0.0
    A2[0, 0] = 1.0
    b = r.ravel().copy()
    b[0] = psi.ravel()[0]
    ref = spla.spsolve(A2.tocsr(), b)
    np.testing.assert_allclose(psi.ravel(), ref, atol=1e-10)


def test_periodic_sine_mode_exact():
    """r = sin(m x) gives psi = -sin(m x) / lambda(m) (Reading 9 eigenvalues)."""
    g = grid(24, 12, 8, False)
    for m in (1, 3, 11):
        r = np.broadcast_to(np.sin(m * g.xc()), g.shape).copy()
        psi = oracle.solve_poisson(r, g)
        lam = (2 - 2 * np.cos(m * g.dx)) / g.dx ** 2
        np.testing.assert_allclose(psi, -r / lam, atol=1e-13)


def test_wall_neumann_cosine_mode_exact():
    """With walls, cos(pi m (j + 1/2)/ny) are the eigenvectors of the Neumann
    tridiagonal operator with eigenvalue (2 - 2 cos(pi m/ny))/dy^2."""
    g = grid(8, 16, 6, True)
    j = np.arange(g.ny)
    for m, kx in ((1, 0), (3, 2), (7, 1)):
        prof = np.cos(np.pi * m * (j + 0.5) / g.ny)[None, :, None]
        r = np.broadcast_to(prof * np.cos(kx * g.xc()), g.shape).copy()
        psi = oracle.solve_poisson(r, g)
        lam = (2 - 2 * np.cos(np.pi * m / g.ny)) / g.dy ** 2 + (2 - 2 * np.cos(kx * g.dx)) / g.dx ** 2
        diff = psi + r / lam
        # exact up to the additive constant of the pinned (kx, kz) = (0, 0) system
        assert np.ptp(diff) < 1e-12
        if kx != 0:
            assert np.abs(diff).max() < 1e-12


def test_thomas_matches_banded_solver():
    rng = np.random.default_rng(2)
    n = 13
    lo, up = rng.uniform(0.5, 1, n), rng.uniform(0.5, 1, n)
    d = -(lo + up) - rng.uniform(0.1, 1, n)
    lo[0] = 0.0
    up[-1] = 0.0
    rhs = rng.standard_normal(n)
    x = thomas(lo, d, up, rhs)
    ab = np.zeros((3, n))
    ab[0, 1:] = up[:-1]
    ab[1] = d
    ab[2, :-1] = lo[1:]
    np.testing.assert_allclose(x, solve_banded((1, 1), ab, rhs), atol=1e-13)


@pytest.mark.parametrize("walls", [False, True])
def test_projection_divergence_below_1e12(walls):
    """Spec bound: after one FP64 projection max|div u| <= 1e-12."""
    geo = inputs.geometry(32, 24, 16, 2 * np.pi, 2.0 if walls else 2 * np.pi, 2 * np.pi, walls)
    g = oracle.Grid(32, 24, 16, geo['lx'], geo['ly'], geo['lz'], walls)
    rng = np.random.default_rng(7)
    U, V, W = (rng.standard_normal(g.shape) for _ in range(3))
    if walls:
        V[:, -1] = 0.0
    U2, V2, W2, psi = oracle.project(U, V, W, g, 1.0)
    assert np.abs(oracle.divergence(U2, V2, W2, g)).max() <= 1e-12
    # projecting a solenoidal field changes it only by round-off
    U3, V3, W3, _ = oracle.project(U2, V2, W2, g, 1.0)
    assert max(np.abs(U3 - U2).max(), np.abs(V3 - V2).max(), np.abs(W3 - W2).max()) < 1e-12


def test_eigenvalues_match_discrete_laplacian_of_plane_wave():
    n, h = 12, 0.3
    lam = eigenvalues(n, h)
    x = np.arange(n)
    for m in range(n):
        e = np.exp(2j * np.pi * m * x / n)
        lap = (np.roll(e, -1) - 2 * e + np.roll(e, 1)) / h ** 2
        np.testing.assert_allclose(lap, -lam[m] * e, atol=1e-12)
