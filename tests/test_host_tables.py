"""Host-side Thomas tables (no GPU): the FP64 pivot tables that the wall-normal
solves sweep, built by the library's host code, checked against dense solves of
the tridiagonal systems written out from their definition; and the
double-single form of single-precision states (each double as hi + lo floats).

A small program compiled by nvcc against the library's internal header (which
also holds device code) prints the tables on the host; the checks run here in
numpy.  No GPU is needed: the program makes no CUDA call."""

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_1803_09563_gb300', 'csrc')

PROGRAM = r'''
#include <cstdio>
#include <vector>
#include "evp_internal.cuh"
using namespace evp;
int main(int argc, char** argv) {
    const int ny = 7, nz = 4, nxh = 3;
    const double dy = 0.3, c = 0.05;
    std::vector<double> lx = {0.0, 1.5, 4.0};
    std::vector<double> lz = {0.0, 2.0, 3.5};                  // nz/2 + 1 entries
    std::vector<double> T = thomas_table(ny, nz, nxh, dy, lx, lz);
    std::vector<double> Hu = helmholtz_table(ny, nz, nxh, dy, lx, lz, c, false);
    std::vector<double> Hv = helmholtz_table(ny, nz, nxh, dy, lx, lz, c, true);
    std::vector<float> F = thomas_table_ds(T);
    for (double v : T) std::printf("%.17g\n", v);
    for (double v : Hu) std::printf("%.17g\n", v);
    for (double v : Hv) std::printf("%.17g\n", v);
    for (float v : F) std::printf("%.9g\n", (double)v);
    return 0;
}
'''
NY, NZ, NXH, DY, C = 7, 4, 3, 0.3, 0.05
LX = [0.0, 1.5, 4.0]
LZ = [0.0, 2.0, 3.5]


@pytest.fixture(scope='module')
def tables(tmp_path_factory):
    from paper_1803_09563_gb300 import build
    nvcc = build.nvcc()
    if shutil.which(nvcc) is None:
        pytest.skip('needs nvcc')
    d = tmp_path_factory.mktemp('tables')
    src = d / 'tables.cu'
    src.write_text(PROGRAM)
    exe = d / 'tables'
    subprocess.run([nvcc, '-std=c++17', '-O1', '-I', CSRC, '-I', os.path.join(ROOT, 'include'), str(src),
                    '-o', str(exe)], check=True)
    vals = np.array([float(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                                      check=True).stdout.split()])
    n = (NZ // 2 + 1) * NY * NXH * 2
    T, Hu, Hv, F = vals[:n], vals[n:2 * n], vals[2 * n:3 * n], vals[3 * n:]
    # nine significant digits identify a float exactly: back to the float's value
    F = F.astype(np.float32).astype(np.float64)
    shape = (NZ // 2 + 1, NY, NXH, 2)
    return T.reshape(shape), Hu.reshape(shape), Hv.reshape(shape), F.reshape(shape[:3] + (4,))


def solve_with_table(P, r, lo):
    """The recurrence the kernels run with a table's pivots (m_j, c'_j) and the
    constant sub-diagonal lo: d'_j = (r_j - lo d'_{j-1}) m_j, then
    x_j = d'_j - c'_j x_{j+1}."""
    n = len(r)
    d = np.zeros(n)
    for j in range(n):
        d[j] = (r[j] - (lo * d[j - 1] if j > 0 else 0.0)) * P[j, 0]
    x = np.zeros(n)
    x[-1] = d[-1]
    for j in range(n - 2, -1, -1):
        x[j] = d[j] - P[j, 1] * x[j + 1]
    return x


def poisson_matrix(lm, pinned):
    """Rows idy2 x_{j-1} - (2 idy2 + lm) x_j + idy2 x_{j+1}; Neumann ends (the
    ghost equals the boundary value, so the end rows lose one idy2); the pinned
    system replaces row 0 by x_0 = r_0."""
    i2 = 1.0 / DY ** 2
    A = np.zeros((NY, NY))
    for j in range(NY):
        A[j, j] = -2 * i2 - lm
        if j > 0:
            A[j, j - 1] = i2
        else:
            A[j, j] += i2
        if j < NY - 1:
            A[j, j + 1] = i2
        else:
            A[j, j] += i2
    if pinned:
        A[0, :] = 0.0
        A[0, 0] = 1.0
    return A


def helmholtz_matrix(lm, kind_v):
    """x - c lap(x) = r along y: rows -cy x_{j-1} + (1 + c lm + 2 cy) x_j - cy x_{j+1};
    u, w (centred): odd no-slip mirror, the ghost is minus the boundary value;
    v (faces): zero faces beyond rows 0 .. ny-2, row ny-1 (the wall face) x = 0."""
    cy = C / DY ** 2
    A = np.zeros((NY, NY))
    m = NY - 1 if kind_v else NY
    for j in range(m):
        A[j, j] = 1 + C * lm + 2 * cy
        if j > 0:
            A[j, j - 1] = -cy
        elif not kind_v:
            A[j, j] += cy
        if j < m - 1:
            A[j, j + 1] = -cy
        elif not kind_v:
            A[j, j] += cy
    if kind_v:
        A[NY - 1, NY - 1] = 1.0
    return A


def test_poisson_pivot_table_solves_the_systems(tables):
    T = tables[0]
    rng = np.random.default_rng(3)
    for kz in range(NZ // 2 + 1):
        for kx in range(NXH):
            pinned = kx == 0 and kz == 0
            A = poisson_matrix(LX[kx] + LZ[kz], pinned)
            r = rng.standard_normal(NY)
            if pinned:
                r[0] = 0.0
            x = solve_with_table(T[kz, :, kx, :], r, 1.0 / DY ** 2)
            ref = np.linalg.solve(A, r)
            assert np.allclose(x, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), (kz, kx)


@pytest.mark.parametrize("kind_v", [False, True])
def test_helmholtz_pivot_tables_solve_the_systems(tables, kind_v):
    H = tables[2 if kind_v else 1]
    rng = np.random.default_rng(4)
    for kz in range(NZ // 2 + 1):
        for kx in range(NXH):
            A = helmholtz_matrix(LX[kx] + LZ[kz], kind_v)
            r = rng.standard_normal(NY)
            x = solve_with_table(H[kz, :, kx, :], r, -C / DY ** 2)
            if kind_v:
                r = r.copy()
                r[-1] = 0.0          # the wall face's solution is zero whatever its right-hand side
                assert x[-1] == 0.0
            ref = np.linalg.solve(A, r)
            assert np.allclose(x, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), (kz, kx, kind_v)


def test_double_single_table_reproduces_the_doubles(tables):
    """hi is the double rounded to float and hi + lo recovers the double to about
    2^-48 of its size (the remainder rounded to float)."""
    T, F = tables[0], tables[3]
    for q in range(2):
        d = T[..., q]
        hi = F[..., 2 * q]
        lo = F[..., 2 * q + 1]
        assert np.array_equal(hi, d.astype(np.float32).astype(np.float64))
        err = np.abs((hi + lo) - d)
        assert np.all(err <= 2.0 ** -47 * np.abs(d) + 1e-300)
    # the pinned system's row 0 (m = 1, c' = 0) and every system's last c' (0) are exact
    assert F[0, 0, 0, 0] == 1.0 and F[0, 0, 0, 1] == 0.0
    assert np.all(F[:, -1, :, 2] == 0.0) and np.all(F[:, -1, :, 3] == 0.0)
