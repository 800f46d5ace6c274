"""The bounds-checked build (``build.py --debug`` -> libevp_debug.so, -DEVP_DEBUG).

In that build the stress and momentum kernels check every staged copy (source
inside one of the kernel's fields, destination inside its shared-memory staging
area, 16-byte alignment of 16-byte copies) and fill the staging area with NaN
bytes before each tile, so that a stencil reading a value no copy wrote gives a
non-finite result.  A failed check skips the copy and makes evp_sync return
EVP_ERR_BOUNDS; nothing traps.

The test runs the same cases through both libraries in child processes (the
binding loads the library that EVP_LIB names): RK3 steps of every model with and
without walls, on grids that take the 16-byte and the element-wise staging, the
right-hand-side mode, artificial diffusion, soft particles, a two-phase AB2
state and a batch of members on three grids.  Every case must report no failed
check and give the release library's fields bit for bit (the checks change no
arithmetic, and no NaN from the poisoned staging reaches an output)."""

import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    from paper_1803_09563_gb300 import evp, inputs
    out, codes = {}, {}

    def fields(sim):
        fs = [evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P]
        if sim.model != evp.EVP_NEWTONIAN:
            fs += [evp.EVP_BXX + c for c in range(6)]
        return {f: sim.get(f) for f in fs}

    def record(name, sim):
        name = name.replace('/', '.').replace(' ', '').replace('(', '').replace(')', '').replace(',', '_')
        code, bits, _ = sim.sync(raise_on_error=False, max_div=False)
        codes[name] = (code, bits)
        for f, arr in fields(sim).items():
            out[f'{name}.{f}'] = arr

    def make(shape, model, precision, seed=3, **extra):
        nx, ny, nz, walls = shape
        ly = 2.0 if walls else 2 * np.pi
        geo = inputs.geometry(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
        U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, seed, 3), 1.0)
        B = inputs.spd_conformation(geo, seed + 1, amp=0.4)
        if walls:
            V = V.copy()
            V[:, -1] = 0.0
        sim = evp.Simulation(evp.make_grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls), model,
                             evp.make_params(Re=2.0, Wi=0.8, beta=0.4, precision=precision, **extra))
        sim.set_state(U, V, W, None, None if model == 'newtonian' else B)
        return sim, geo

    models = [('newtonian', {}), ('oldroyd_b', {}), ('fene_p', {'L2': 60.0}), ('saramito', {'Bi': 0.3}),
              ('neo_hookean', {})]
    # 48 and 36 columns stage in 16-byte chunks in FP32, 18 element by element
    shapes = [(48, 24, 16, False), (36, 20, 16, True), (18, 12, 12, True)]
    for prec in (evp.EVP_FP32, evp.EVP_FP64):
        for shape in shapes:
            for model, extra in models:
                sim, _ = make(shape, model, prec, **extra)
                for _ in range(2):
                    sim.step(2e-3)
                record(f'rk3/{prec}/{shape}/{model}', sim)
                sim.close()
        # right-hand side mode of the stress kernel
        import torch
        sim, _ = make((36, 20, 16, True), 'saramito', prec, Bi=0.3)
        rt = torch.empty((6,) + sim.shape, dtype=sim.dtype, device='cuda')
        evp.evp_stress_rhs(sim.handle, rt)
        record(f'rhs/{prec}', sim)
        out[f'rhs.{prec}.rt'] = rt.cpu().numpy()
        sim.close()
        # local artificial diffusion
        sim, _ = make((48, 24, 16, False), 'fene_p', prec, L2=60.0, art_diff=1e-3)
        for _ in range(2):
            sim.step(2e-3)
        record(f'diff/{prec}', sim)
        sim.close()
        # soft particles (neo-Hookean, the stress built in the momentum kernel)
        sim, geo = make((36, 20, 16, True), 'neo_hookean', prec, soft_particles=1)
        d = inputs.sphere_distance(geo, (3.0, 0.0, 3.0), 0.6)
        sim.set(evp.EVP_PHI, 0.5 * (1.0 - np.tanh(d / 0.2)))
        for _ in range(2):
            sim.step(2e-3)
        record(f'soft/{prec}', sim)
        sim.close()
        # two-phase AB2 state (the stress kernel reads the Heaviside)
        n, L = 24, 2.0
        grid = evp.make_grid(n, n, n, L, L, L, walls_y=True)
        prm = evp.make_params(Re=10.0, Wi=0.5, beta=0.5, Bi=0.3, precision=prec, integrator=evp.EVP_AB2,
                              sigma=0.1, drho_g=1.0, reinit_every=0)
        sim = evp.Simulation(grid, 'saramito', prm)
        g2 = inputs.geometry(n, n, n, L, L, L, True)
        sim.set(evp.EVP_PHI, inputs.sphere_distance(g2, (1.0, 0.0, 1.0), 0.4))
        for _ in range(2):
            sim.step(1e-3)
        record(f'ab2/{prec}', sim)
        sim.close()
        # a batch of members on three grids (persistent stress and momentum kernels)
        batch = evp.Batch(prec)
        members = [make(s, m, prec, seed=7 + q, **e)[0] for q, (s, (m, e)) in
                   enumerate(zip(shapes, models[1:4]))]
        for m in members:
            batch.admit(m, 2e-3)
        for _ in range(2):
            batch.step()
        for q, m in enumerate(members):
            batch.evict(m)
            record(f'batch/{prec}/{q}', m)
            m.close()
        batch.close()
    return out, codes


def _run(lib, path):
    env = dict(os.environ, EVP_LIB=lib)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), path], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


@pytest.mark.gpu
def test_debug_build_reports_no_failed_check_and_matches_release(tmp_path):
    sys.path.insert(0, ROOT)
    from paper_1803_09563_gb300 import build, evp
    rel = build.build()
    dbg = build.build(debug=True)
    _run(rel, str(tmp_path / 'rel.npz'))
    _run(dbg, str(tmp_path / 'dbg.npz'))
    R = np.load(tmp_path / 'rel.npz', allow_pickle=True)
    D = np.load(tmp_path / 'dbg.npz', allow_pickle=True)
    codes_r, codes_d = R['__codes__'].item(), D['__codes__'].item()
    assert set(codes_r) == set(codes_d) and len(codes_d) > 40
    for name, (code, bits) in codes_d.items():
        assert code == evp.EVP_OK and bits == 0, (name, code, bits)
        assert codes_r[name] == (code, bits), name
    keys = [k for k in R.files if k != '__codes__']
    assert set(keys) == set(D.files) - {'__codes__'}
    for k in keys:
        a, b = R[k], D[k]
        assert np.all(np.isfinite(b)), k
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), k


if __name__ == '__main__':
    sys.path.insert(0, ROOT)
    arrays, codes = _cases()
    np.savez(sys.argv[1], __codes__=np.array(codes, dtype=object), **arrays)
