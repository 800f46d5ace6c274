"""Thin ctypes binding of libevp (include/evp.h).  Argument marshalling only:
every step of the time step runs in the library's CUDA kernels.  There is no
fallback -- if libevp.so is missing or cannot be loaded, ``load()`` raises.

The functions keep the C names (``evp_init``, ``evp_step``, ...).  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays; device tensors are passed by
pointer (``on_device=1``), host arrays by host pointer.
"""

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_longlong, c_size_t, c_uint, c_ulonglong, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# EVP_LIB selects another in-tree build of the library (the bounds-checked
# libevp_debug.so of ``build.py --debug``)
LIB_PATH = os.environ.get('EVP_LIB') or os.path.join(HERE, 'libevp.so')

# evp_status
EVP_OK, EVP_ERR_ARG, EVP_ERR_OOM, EVP_ERR_CUDA, EVP_ERR_NONFINITE, EVP_ERR_UNPHYSICAL, EVP_ERR_TIMEOUT, \
    EVP_ERR_STATE, EVP_ERR_BOUNDS = range(9)
EVP_BIT_NONFINITE, EVP_BIT_TRACE_LIMIT, EVP_BIT_DET_NEG, EVP_BIT_BOUNDS = 0x1, 0x2, 0x4, 0x8
# evp_model
EVP_NEWTONIAN, EVP_OLDROYD_B, EVP_FENE_P, EVP_SARAMITO, EVP_NEO_HOOKEAN = range(5)
MODEL_IDS = {'newtonian': 0, 'oldroyd_b': 1, 'fene_p': 2, 'saramito': 3, 'neo_hookean': 4}
EVP_FP64, EVP_FP32 = 0, 1
EVP_RK3, EVP_AB2 = 0, 1
EVP_BATCH_MAX = 64   # members of one batch
# evp_field
EVP_U, EVP_V, EVP_W, EVP_P = 0, 1, 2, 3
EVP_BXX, EVP_BXY, EVP_BXZ, EVP_BYY, EVP_BYZ, EVP_BZZ = range(4, 10)
EVP_RT_XX = 10
EVP_NH_X = 16
EVP_PSI = 19
EVP_PHI = 20
EVP_SOLID_X, EVP_SOLID_Y, EVP_SOLID_Z = 21, 22, 23


class evp_grid(ctypes.Structure):
    _fields_ = [('nx', c_int), ('ny', c_int), ('nz', c_int), ('lx', c_double), ('ly', c_double),
                ('lz', c_double), ('walls_y', c_int)]


class evp_params(ctypes.Structure):
    _fields_ = [('Re', c_double), ('Wi', c_double), ('beta', c_double), ('Bi', c_double), ('L2', c_double),
                ('bi_def', c_int), ('dpdx', c_double), ('abc_amp', c_double), ('abc_k', c_double),
                ('precision', c_int), ('integrator', c_int), ('mu_ratio', c_double), ('ls_eps_cells', c_double),
                ('sigma', c_double), ('drho_g', c_double), ('reinit_every', c_int), ('reinit_iters', c_int),
                ('rho_ratio', c_double), ('gravity', c_double), ('penalization', c_int),
                ('art_diff', c_double), ('ls_mass_iters', c_int), ('viscous_implicit', c_int),
                ('soft_particles', c_int), ('thomas_fp64', c_int), ('reserved', c_double * 4)]


class EvpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f'libevp error {code}: {msg}')
        self.code = code


class evp_tile_config(ctypes.Structure):
    _fields_ = [('stress_kz', c_int), ('momentum_kz', c_int), ('stress_ctas_per_sm', c_int),
                ('momentum_ctas_per_sm', c_int), ('fft_cols', c_int)]

    def as_tuple(self):
        return (self.stress_kz, self.momentum_kz, self.stress_ctas_per_sm, self.momentum_ctas_per_sm, self.fft_cols)


class evp_diag(ctypes.Structure):
    _fields_ = [('kinetic_energy', c_double), ('max_div', c_double), ('min_det_B', c_double),
                ('max_tr_B', c_double), ('max_tr_B_over_L2', c_double), ('yielded_fraction', c_double),
                ('nonfinite_cells', c_ulonglong), ('yielded_cells', c_ulonglong)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def load(path=None):
    """Load libevp.so (built by ``paper_1803_09563_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f'libevp.so not found at {path}: build it with '
                           '`python -c "import __graft_entry__ as g; g.build()"`')
    lib = ctypes.CDLL(path)
    sig = {
        'evp_state_bytes': (c_size_t, [POINTER(evp_grid), c_int, POINTER(evp_params)]),
        'evp_init': (c_int, [POINTER(evp_grid), c_int, POINTER(evp_params), c_void_p, c_void_p, c_size_t,
                             POINTER(c_void_p)]),
        'evp_destroy': (c_int, [c_void_p]),
        'evp_set_field': (c_int, [c_void_p, c_int, c_void_p, c_int]),
        'evp_get_field': (c_int, [c_void_p, c_int, c_void_p, c_int]),
        'evp_set_fields': (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_void_p), c_int]),
        'evp_get_fields': (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_void_p), c_int]),
        'evp_step': (c_int, [c_void_p, c_double]),
        'evp_step_io': (c_int, [c_void_p, c_double, c_int, POINTER(c_int), POINTER(c_void_p), c_int, POINTER(c_int),
                                POINTER(c_void_p)]),
        'evp_set_graph': (c_int, [c_void_p, c_int]),
        'evp_set_pdl': (c_int, [c_void_p, c_int]),
        'evp_set_nvtx': (c_int, [c_void_p, c_int]),
        'evp_set_particles': (c_int, [c_void_p, c_int, c_void_p, c_int]),
        'evp_get_particles': (c_int, [c_void_p, c_int, c_void_p]),
        'evp_substep': (c_int, [c_void_p, c_double, c_int]),
        'evp_project': (c_int, [c_void_p]),
        'evp_poisson_solve': (c_int, [c_void_p, c_void_p, c_void_p]),
        'evp_stress_rhs': (c_int, [c_void_p, c_void_p]),
        'evp_poisson_solve_static': (c_int, [POINTER(evp_grid), c_int, c_void_p, c_void_p, c_void_p]),
        'evp_sync': (c_int, [c_void_p, POINTER(c_uint), POINTER(c_double)]),
        'evp_diagnostics': (c_int, [c_void_p, POINTER(evp_diag)]),
        'evp_selftest': (c_int, [POINTER(c_ulonglong)]),
        'evp_fma_peak': (c_int, [c_int, POINTER(c_double)]),
        'evp_batch_create': (c_int, [c_int, c_size_t, c_void_p, POINTER(c_void_p)]),
        'evp_batch_admit': (c_int, [c_void_p, c_void_p, c_double]),
        'evp_batch_evict': (c_int, [c_void_p, c_void_p]),
        'evp_batch_step': (c_int, [c_void_p]),
        'evp_batch_info': (c_int, [c_void_p, POINTER(c_int), POINTER(c_size_t)]),
        'evp_batch_set_graph': (c_int, [c_void_p, c_int]),
        'evp_batch_destroy': (c_int, [c_void_p]),
        'evp_tune': (c_int, [POINTER(evp_grid), c_int, POINTER(evp_params), c_int, POINTER(evp_tile_config),
                             POINTER(c_double), POINTER(c_int)]),
        'evp_tile_time': (c_int, [POINTER(evp_grid), c_int, POINTER(evp_params), POINTER(evp_tile_config), c_int,
                                  POINTER(c_double)]),
        'evp_tile_config_get': (c_int, [POINTER(evp_grid), c_int, c_int, POINTER(evp_tile_config)]),
        'evp_tile_config_set': (c_int, [POINTER(evp_grid), c_int, c_int, POINTER(evp_tile_config)]),
        'evp_kernel_timing': (c_int, [c_void_p, c_int]),
        'evp_kernel_times': (c_int, [c_void_p, POINTER(c_double), POINTER(c_longlong), c_int]),
        'evp_kernel_name': (c_char_p, [c_int]),
        'evp_num_kernels': (c_int, []),
        'evp_last_error': (c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/evp.h that the binding resolves."""
    return ['evp_state_bytes', 'evp_init', 'evp_destroy', 'evp_set_field', 'evp_get_field', 'evp_step',
            'evp_substep', 'evp_project', 'evp_poisson_solve', 'evp_stress_rhs', 'evp_sync', 'evp_kernel_timing',
            'evp_kernel_times', 'evp_kernel_name', 'evp_num_kernels', 'evp_last_error', 'evp_poisson_solve_static',
            'evp_set_graph', 'evp_selftest', 'evp_set_pdl', 'evp_set_particles', 'evp_get_particles',
            'evp_set_fields', 'evp_get_fields', 'evp_fma_peak', 'evp_batch_create', 'evp_batch_admit',
            'evp_batch_evict', 'evp_batch_step', 'evp_batch_info', 'evp_batch_set_graph', 'evp_batch_destroy',
            'evp_tune', 'evp_tile_time', 'evp_tile_config_get', 'evp_tile_config_set', 'evp_step_io',
            'evp_diagnostics', 'evp_set_nvtx']


def _check(code):
    if code != EVP_OK:
        raise EvpError(code, load().evp_last_error().decode())
    return code


def _ptr(a):
    """(pointer, on_device, nbytes) of a torch tensor or numpy array (contiguous)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            assert a.is_contiguous()
            if a.is_cuda and not torch.cuda.is_current_stream_capturing():
                # the library works on its own stream: finish torch's pending work on
                # the tensor (a stream being captured orders the work by the capture
                # and may not be synchronised)
                torch.cuda.current_stream(a.device).synchronize()
            return a.data_ptr(), int(a.is_cuda), a.numel() * a.element_size()
    except ImportError:
        pass
    assert isinstance(a, np.ndarray) and a.flags['C_CONTIGUOUS']
    return a.ctypes.data, 0, a.nbytes


def make_grid(nx, ny, nz, lx, ly, lz, walls_y=False):
    return evp_grid(int(nx), int(ny), int(nz), float(lx), float(ly), float(lz), int(bool(walls_y)))


def make_params(Re, Wi=1.0, beta=1.0, Bi=0.0, L2=0.0, bi_def=0, dpdx=0.0, abc_amp=0.0, abc_k=0.0,
                precision=EVP_FP64, integrator=EVP_RK3, mu_ratio=1.0, ls_eps_cells=1.5, sigma=0.0, drho_g=0.0,
                reinit_every=10, reinit_iters=3, penalization=0, rho_ratio=0.0, gravity=0.0, art_diff=0.0,
                ls_mass_iters=0, viscous_implicit=0, soft_particles=0, thomas_fp64=0):
    p = evp_params()
    p.Re, p.Wi, p.beta, p.Bi, p.L2 = float(Re), float(Wi), float(beta), float(Bi), float(L2)
    p.bi_def, p.dpdx, p.abc_amp, p.abc_k = int(bi_def), float(dpdx), float(abc_amp), float(abc_k)
    p.precision, p.integrator = int(precision), int(integrator)
    p.mu_ratio, p.ls_eps_cells, p.sigma, p.drho_g = float(mu_ratio), float(ls_eps_cells), float(sigma), float(drho_g)
    p.reinit_every, p.reinit_iters = int(reinit_every), int(reinit_iters)
    p.penalization = int(penalization)
    p.rho_ratio, p.gravity = float(rho_ratio), float(gravity)
    p.art_diff = float(art_diff)
    p.ls_mass_iters = int(ls_mass_iters)
    p.viscous_implicit = int(viscous_implicit)
    p.soft_particles = int(soft_particles)
    p.thomas_fp64 = int(thomas_fp64)
    return p


def evp_state_bytes(grid, model, params):
    return load().evp_state_bytes(ctypes.byref(grid), int(model), ctypes.byref(params))


def evp_init(grid, model, params, stream=None, arena=None, arena_bytes=0):
    h = c_void_p()
    _check(load().evp_init(ctypes.byref(grid), int(model), ctypes.byref(params), stream, arena,
                           arena_bytes, ctypes.byref(h)))
    return h


def evp_destroy(state):
    return _check(load().evp_destroy(state))


def evp_set_field(state, field, src):
    p, dev, _ = _ptr(src)
    return _check(load().evp_set_field(state, int(field), p, dev))


def evp_get_field(state, field, dst):
    p, dev, _ = _ptr(dst)
    return _check(load().evp_get_field(state, int(field), p, dev))


def _field_arrays(fields, bufs):
    if len(fields) != len(bufs):
        raise ValueError('one buffer per field')
    ptrs = [_ptr(b) for b in bufs]
    devs = {d for _, d, _ in ptrs}
    if len(devs) > 1:
        raise ValueError('all buffers on the host or all on the device')
    n = len(fields)
    ids = (c_int * n)(*[int(f) for f in fields])
    ps = (c_void_p * n)(*[p for p, _, _ in ptrs])
    return n, ids, ps, (devs.pop() if devs else 0)


def evp_set_fields(state, fields, srcs):
    """Copy several fields into the state with one synchronisation."""
    n, ids, ps, dev = _field_arrays(fields, srcs)
    return _check(load().evp_set_fields(state, n, ids, ps, dev))


def evp_get_fields(state, fields, dsts):
    """Copy several fields out of the state with one synchronisation."""
    n, ids, ps, dev = _field_arrays(fields, dsts)
    return _check(load().evp_get_fields(state, n, ids, ps, dev))


def evp_step(state, dt):
    return _check(load().evp_step(state, float(dt)))


class StepIO:
    """Marshalled argument arrays of evp_step_io for fixed host buffers (built
    once, reused every step; the buffers are numpy arrays or CPU tensors, pinned
    for asynchronous copies)."""

    def __init__(self, in_fields, in_bufs, out_fields, out_bufs):
        self.n_in, self.in_ids, self.in_ps, dev_in = _field_arrays(in_fields, in_bufs)
        self.n_out, self.out_ids, self.out_ps, dev_out = _field_arrays(out_fields, out_bufs)
        if dev_in or dev_out:
            raise ValueError('evp_step_io copies from and to host buffers')
        self.keep = (in_bufs, out_bufs)


def evp_step_io(state, dt, io):
    """One step with host inputs and outputs (see StepIO), enqueued on the state's
    stream without waiting."""
    return _check(load().evp_step_io(state, float(dt), io.n_in, io.in_ids, io.in_ps, io.n_out, io.out_ids,
                                     io.out_ps))


def evp_set_graph(state, enable):
    return _check(load().evp_set_graph(state, int(bool(enable))))


def evp_set_pdl(state, enable):
    return _check(load().evp_set_pdl(state, int(bool(enable))))


def evp_set_nvtx(state, enable):
    """NVTX ranges around steps, substeps and directly launched kernels."""
    return _check(load().evp_set_nvtx(state, int(bool(enable))))


def evp_set_particles(state, particles, iters=3):
    """``particles``: sequence of (centre (3), radius, velocity (3), angular velocity (3)
    [, density ratio rho_p/rho_f: 0 or absent = prescribed motion])."""
    rows = []
    for q in particles:
        c, r, u, w = q[:4]
        dens = q[4] if len(q) > 4 else 0.0
        rows.append(list(c) + [r] + list(u) + list(w) + [dens])
    desc = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1))
    n = len(particles)
    return _check(load().evp_set_particles(state, n, desc.ctypes.data if n else None, int(iters)))


def evp_get_particles(state, n):
    """(n, 15) array: centre, velocity, angular velocity, force and torque on each
    particle (the last two from the last substep)."""
    out = np.zeros((max(n, 1), 15), dtype=np.float64)
    _check(load().evp_get_particles(state, n, out.ctypes.data))
    return out[:n]


def evp_substep(state, dt, k):
    return _check(load().evp_substep(state, float(dt), int(k)))


def evp_project(state):
    return _check(load().evp_project(state))


def evp_poisson_solve(state, rhs, psi):
    return _check(load().evp_poisson_solve(state, _ptr(rhs)[0], _ptr(psi)[0]))


def evp_poisson_solve_static(grid, precision, rhs, psi, stream=None):
    """The no-allocation Poisson solve (static device scratch; see evp.h)."""
    return _check(load().evp_poisson_solve_static(ctypes.byref(grid), int(precision), _ptr(rhs)[0], _ptr(psi)[0],
                                                  stream))


def evp_stress_rhs(state, rt):
    return _check(load().evp_stress_rhs(state, _ptr(rt)[0]))


def evp_sync(state, raise_on_error=True, max_div=True):
    """Returns (code, status bits, FP64 max |div u| of the current velocity, which
    after a step is the last projection's output; None with max_div=False, when
    no residual kernel runs)."""
    bits = c_uint(0)
    md = c_double(0.0)
    code = load().evp_sync(state, ctypes.byref(bits), ctypes.byref(md) if max_div else None)
    if raise_on_error and code not in (EVP_OK,):
        _check(code)
    return code, bits.value, md.value if max_div else None


def evp_diagnostics(state):
    """Monitoring quantities of the current state as a dict (evp_diag of evp.h)."""
    d = evp_diag()
    _check(load().evp_diagnostics(state, ctypes.byref(d)))
    return d.as_dict()


def evp_fma_peak(precision):
    """Measured plain-FMA peak of the current device in FLOP/s (EVP_FP32: packed
    f32x2 FMAs; EVP_FP64: double FMAs)."""
    r = c_double(0.0)
    _check(load().evp_fma_peak(int(precision), ctypes.byref(r)))
    return r.value


def evp_batch_create(precision, budget_bytes=0, stream=None):
    h = c_void_p()
    _check(load().evp_batch_create(int(precision), int(budget_bytes), stream, ctypes.byref(h)))
    return h


def evp_batch_admit(batch, state, dt):
    return _check(load().evp_batch_admit(batch, state, float(dt)))


def evp_batch_evict(batch, state):
    return _check(load().evp_batch_evict(batch, state))


def evp_batch_step(batch):
    return _check(load().evp_batch_step(batch))


def evp_batch_info(batch):
    """(members, bytes admitted)"""
    n, b = c_int(0), c_size_t(0)
    _check(load().evp_batch_info(batch, ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def evp_batch_set_graph(batch, enable):
    return _check(load().evp_batch_set_graph(batch, int(bool(enable))))


def evp_batch_destroy(batch):
    return _check(load().evp_batch_destroy(batch))


def evp_tune(grid, model, params, exhaustive=False):
    """(config, ms per step, trials) chosen by the library's autotuner for this grid."""
    cfg, ms, n = evp_tile_config(), c_double(0.0), c_int(0)
    m = MODEL_IDS[model] if isinstance(model, str) else int(model)
    _check(load().evp_tune(ctypes.byref(grid), m, ctypes.byref(params), int(bool(exhaustive)), ctypes.byref(cfg),
                           ctypes.byref(ms), ctypes.byref(n)))
    return cfg, ms.value, n.value


def evp_tile_time(grid, model, params, cfg, steps=20):
    ms = c_double(0.0)
    m = MODEL_IDS[model] if isinstance(model, str) else int(model)
    if not isinstance(cfg, evp_tile_config):
        cfg = evp_tile_config(*cfg)
    _check(load().evp_tile_time(ctypes.byref(grid), m, ctypes.byref(params), ctypes.byref(cfg), int(steps),
                                ctypes.byref(ms)))
    return ms.value


def evp_tile_config_get(grid, precision, model):
    cfg = evp_tile_config()
    m = MODEL_IDS[model] if isinstance(model, str) else int(model)
    _check(load().evp_tile_config_get(ctypes.byref(grid), int(precision), m, ctypes.byref(cfg)))
    return cfg


def evp_tile_config_set(grid, precision, model, cfg):
    m = MODEL_IDS[model] if isinstance(model, str) else int(model)
    if not isinstance(cfg, evp_tile_config):
        cfg = evp_tile_config(*cfg)
    return _check(load().evp_tile_config_set(ctypes.byref(grid), int(precision), m, ctypes.byref(cfg)))


def evp_selftest():
    """Failures of the integer-operation FP32 <-> FP64 conversions against the
    device's conversion instructions (0 expected)."""
    bad = c_ulonglong(0)
    _check(load().evp_selftest(ctypes.byref(bad)))
    return bad.value


def evp_kernel_timing(state, enable):
    return _check(load().evp_kernel_timing(state, int(bool(enable))))


def evp_kernel_times(state):
    """{kernel name: (total ms, launches)} since the last call (synchronises)."""
    lib = load()
    n = lib.evp_num_kernels()
    ms = (c_double * n)()
    cnt = (c_longlong * n)()
    _check(lib.evp_kernel_times(state, ms, cnt, n))
    return {lib.evp_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(n)}


def evp_last_error():
    return load().evp_last_error().decode()


class Simulation:
    """Owns one libevp state; fields move as numpy float64 arrays (converted to the
    state's precision) or as CUDA tensors of that precision."""

    def __init__(self, grid, model, params, stream=None):
        import torch
        self.grid, self.params = grid, params
        self.model = MODEL_IDS[model] if isinstance(model, str) else int(model)
        self.shape = (grid.nz, grid.ny, grid.nx)
        self.dtype = torch.float32 if params.precision == EVP_FP32 else torch.float64
        self.np_dtype = np.float32 if params.precision == EVP_FP32 else np.float64
        self.handle = evp_init(grid, self.model, params, stream)

    def close(self):
        if self.handle is not None:
            evp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, field, arr):
        import torch
        if isinstance(arr, torch.Tensor):
            t = arr.to(self.dtype).contiguous()
        else:
            t = np.ascontiguousarray(np.asarray(arr, dtype=self.np_dtype).reshape(self.shape))
        evp_set_field(self.handle, field, t)

    def get(self, field, device=False):
        import torch
        if device:
            out = torch.empty(self.shape, dtype=self.dtype, device='cuda')
        else:
            out = np.empty(self.shape, dtype=self.np_dtype)
        evp_get_field(self.handle, field, out)
        return out

    def set_state(self, U=None, V=None, W=None, p=None, B=None):
        for f, a in ((EVP_U, U), (EVP_V, V), (EVP_W, W), (EVP_P, p)):
            if a is not None:
                self.set(f, a)
        if B is not None:
            for c in range(6):
                self.set(EVP_BXX + c, B[c])

    def step(self, dt):
        evp_step(self.handle, dt)

    def substep(self, dt, k):
        evp_substep(self.handle, dt, k)

    def project(self):
        evp_project(self.handle)

    def sync(self, raise_on_error=True, max_div=True):
        return evp_sync(self.handle, raise_on_error, max_div)

    def diagnostics(self):
        return evp_diagnostics(self.handle)


class Batch:
    """A libevp batch: member Simulations advance together, one RK3 step of each
    member's dt per ``step()``."""

    def __init__(self, precision, budget_bytes=0, stream=None):
        self.handle = evp_batch_create(precision, budget_bytes, stream)
        self.members = []

    def admit(self, sim, dt):
        evp_batch_admit(self.handle, sim.handle, dt)
        self.members.append(sim)

    def evict(self, sim):
        evp_batch_evict(self.handle, sim.handle)
        self.members.remove(sim)

    def step(self):
        evp_batch_step(self.handle)

    def info(self):
        return evp_batch_info(self.handle)

    def close(self):
        if self.handle is not None:
            evp_batch_destroy(self.handle)
            self.handle = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
