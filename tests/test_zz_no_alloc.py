"""The no-allocation Poisson entry point, evp_poisson_solve_static, for callers
that cannot allocate device memory (stream capture, host frameworks that own
all device memory, fixed memory budgets).  It keeps its scratch in a static
8 MiB device array; it must give the result of the state-owning
evp_poisson_solve, call after call, and reject grids too large for the array.

Collected last on purpose: a failure here comes after every other test ran.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the tolerances of the Poisson parity tests (relative, per field)
TOL = {0: 1e-12, 1: 2e-6}


def rel(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def state_solve(evp, grid, prec, r):
    """Reference: the existing entry point with a library-allocated state."""
    import torch
    dt = torch.float32 if prec else torch.float64
    sim = evp.Simulation(grid, 'newtonian', evp.make_params(Re=1.0, precision=prec))
    rd = torch.tensor(r, dtype=dt, device='cuda')
    out = torch.empty_like(rd)
    evp.evp_poisson_solve(sim.handle, rd, out)
    sim.sync()
    res = out.cpu().numpy().astype(np.float64)
    sim.close()
    return res


def static_solve(evp, grid, prec, r):
    import torch
    dt = torch.float32 if prec else torch.float64
    rd = torch.tensor(r, dtype=dt, device='cuda')
    out = torch.full_like(rd, float('nan'))
    evp.evp_poisson_solve_static(grid, prec, rd, out, None)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def case(seed, shape):
    nz, ny, nx = shape
    r = np.random.default_rng(seed).standard_normal(shape)
    return r - r.mean()


def test_static_scratch_solve_matches_state_solve(evp):
    walls = evp.make_grid(36, 20, 16, 2 * np.pi, 2.0, 2 * np.pi, True)
    periodic = evp.make_grid(48, 24, 18, 2 * np.pi, 2 * np.pi, 2 * np.pi, False)
    # two calls in a row on the same grid (the array keeps the first call's
    # contents), then a change of grid and precision (tables uploaded again)
    for grid, prec, seed in ((walls, 0, 1), (walls, 0, 2), (periodic, 1, 3), (periodic, 1, 4)):
        r = case(seed, (grid.nz, grid.ny, grid.nx))
        if prec == 1:
            r = r.astype(np.float32).astype(np.float64)
        got = static_solve(evp, grid, prec, r)
        ref = state_solve(evp, grid, prec, r)
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < TOL[prec], (grid.nx, prec, rel(got, ref))


def test_static_scratch_rejects_oversize_grid(evp):
    import torch
    big = evp.make_grid(256, 128, 128, 4 * np.pi, 2.0, 2 * np.pi, True)
    r = torch.zeros((128, 128, 256), dtype=torch.float32, device='cuda')
    with pytest.raises(evp.EvpError) as e:
        evp.evp_poisson_solve_static(big, evp.EVP_FP32, r, r, None)
    assert e.value.code == evp.EVP_ERR_ARG
    assert 'too large' in str(e.value)


def test_static_scratch_solve_in_a_captured_graph(evp):
    """The use the entry point exists for: after one call on the grid (tables in
    the array), a second call on the same grid made while a stream is captured
    into a CUDA graph.  The capture succeeds (no allocation, synchronisation or
    table upload inside it) and the replayed graph gives the state solve's result,
    twice in a row."""
    import torch
    grid = evp.make_grid(36, 20, 16, 2 * np.pi, 2.0, 2 * np.pi, True)
    prec = 0
    r = case(5, (grid.nz, grid.ny, grid.nx))
    ref = state_solve(evp, grid, prec, r)
    rd = torch.tensor(r, dtype=torch.float64, device='cuda')
    out = torch.full_like(rd, float('nan'))
    static_solve(evp, grid, prec, case(6, (grid.nz, grid.ny, grid.nx)))    # warm call on this grid
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    # torch captures in the global mode, where a cudaMalloc, a synchronisation or a
    # pageable copy inside the call would invalidate the capture and raise here
    with torch.cuda.graph(g, stream=side, capture_error_mode='global'):
        evp.evp_poisson_solve_static(grid, prec, rd, out, torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(float('nan'))
        g.replay()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel(got, ref) < TOL[prec], rel(got, ref)
