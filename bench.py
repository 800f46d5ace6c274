"""Benchmark of the EVP time step on GB300.

Workload (default): Saramito EVP channel, 256 x 128 x 128 (x, y, z), periodic in x
and z, no-slip walls at y = +-1, Re = 100, Wi = 1, Bi = 0.5, beta = 0.5, body force
dp/dx = 2/Re, dt = 2e-3, laminar Poiseuille base flow plus a seeded solenoidal
perturbation of max-norm 1e-2 with |k| <= 8.  FP32 fields and stencils, double-single Thomas
sweeps ("FP32-served"), with the same run in FP64 ("FP64 plain") beside it.  The
FP64 divergence residual of the final state is evaluated at sync, after the timed
steps (the steps compute none).

A step is one full RK3 step (three substeps: stress update, momentum predictor,
Poisson solve, projection).  Metric: Mcell-steps/s = cells * steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

N > 1 runs under torchrun, one independent replica per GPU (the time step of one
simulation does not shard); value = cells * steps * N / max-over-ranks time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-steps/s FP32-served vs FP64 plain at stated error; p50/p99 step latency"
WORKLOAD = dict(name="saramito_channel_256x128x128", nx=256, ny=128, nz=128, lx=4 * np.pi, ly=2.0,
                lz=2 * np.pi, walls_y=True, model="saramito", Re=100.0, Wi=1.0, Bi=0.5, beta=0.5,
                dt=2e-3, seed=1, kmax=8, amp=1e-2)


def workload_inputs(w, nz=None):
    from paper_1803_09563_gb300 import inputs
    nz = nz or w['nz']
    lz = w['lz'] * nz / w['nz']
    geo = inputs.geometry(w['nx'], w['ny'], nz, w['lx'], w['ly'], lz, w['walls_y'])
    U, V, W = inputs.poiseuille(geo)
    u2, v2, w2 = inputs.scale_max(*inputs.random_solenoidal(geo, w['seed'], w['kmax']), w['amp'])
    return geo, U + u2, v2, w2


def peaks():
    p = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d['hbm_gbs']), 'measured'
    return 6800.0, 'fallback'


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ('clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,'
         'clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,'
         'clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []          # (host monotonic time, csv line)
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.index), '--query-gpu=' + self.Q,
                                          '--format=csv,noheader,nounits', '-lms', '100'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_first(self, timeout=10.0):
        """Block until nvidia-smi has printed its first sample (its start-up takes
        longer than a short timed region)."""
        t0 = time.monotonic()
        while self.proc is not None and not self.lines and time.monotonic() - t0 < timeout:
            time.sleep(0.02)

    def begin(self):
        self.window = [time.monotonic(), None]

    def end(self):
        self.window[1] = time.monotonic()

    def stop(self, wait_s=3.0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        # a region shorter than the sampling period may hold no sample: wait for the
        # first one printed after it ended (it describes the clocks just after the
        # region, which the region's own work set)
        if self.window is not None and self.window[1] is not None:
            t0 = time.monotonic()
            while (not any(x[0] >= self.window[1] for x in self.lines)
                   and time.monotonic() - t0 < wait_s and self.proc.poll() is None):
                time.sleep(0.02)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        lines = self.lines
        if self.window is not None and self.window[1] is not None:
            inside = [x for x in lines if self.window[0] <= x[0] <= self.window[1]]
            # a region shorter than the sampling period: the first sample after it began
            after = [x for x in lines if x[0] >= self.window[0]][:1]
            self.where = "inside the timed region" if inside else "first sample after the region began"
            lines = inside or after
        for _, l in lines:
            parts = [x.strip() for x in l.split(',')]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == 'active':
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_from": getattr(self, 'where', None)}


def algorithmic_bytes(kernel, w, elt, walls):
    """Minimum bytes each kernel must move per launch, summed over one step's three
    substeps (history read skipped at substep 1, history write skipped at substep 3)."""
    N = w['nx'] * w['ny'] * w['nz']
    nxh = w['nx'] // 2 + 1
    spec = 2 * nxh * w['ny'] * w['nz'] * elt     # complex spectral buffer, bytes
    if kernel == 'stress_weno_update':
        # the method's own words (Eq. rk3tau): read u(3) B(6) [+RT(6)], write B(6)
        # [+RT(6)]: 21, 27, 21.  The summed stress S (6 words written per substep for
        # the momentum step) is the fusion's traffic, counted by fusion_bytes()
        words = (3 + 6 + 6 + 6) + (3 + 6 + 6 + 6 + 6) + (3 + 6 + 6 + 6)
        return words * N * elt, 3
    if kernel == 'momentum_predictor':
        # read u(3) p(1) S(6) [+N(3)], write u*(3) [+N(3)]
        words = (3 + 1 + 6 + 3 + 3) + (3 + 1 + 6 + 3 + 3 + 3) + (3 + 1 + 6 + 3 + 3)
        return words * N * elt, 3
    if kernel == 'div_fft_x':
        return 3 * (3 * N * elt + spec), 3
    if kernel in ('fft_z_forward', 'fft_z_inverse', 'fft_y_modal_solve'):
        return 3 * 2 * spec, 3
    if kernel == 'thomas_y':
        return 3 * 2 * spec, 3
    if kernel == 'ifft_x_psi':
        return 3 * (spec + N * elt), 3
    if kernel == 'project_correct':
        # read u*(3) psi(1) p(1), write u(3) p(1)
        return 3 * 9 * N * elt, 3
    return 0, 1


# Arithmetic of the method counted from its formulas (an FMA counts as two
# operations, a division or square root as one), per cell:
#  stress update, one substep: centre velocity and gradient 48, 18 WENO5
#  reconstructions of 62 (5 differences, 3 candidates 13, smoothness indicators 30,
#  weights and combination 14) = 1116, |u|/h 6, advection sums 12, upper-convected
#  terms 66, Saramito closure 33, source and right-hand side 27, RK3 update 24:
#  1332 in all;
#  whole RK3 step: three times (stress 1332 + momentum predictor about 260 +
#  Poisson chain and correction about 95) = about 5060.
STRESS_FLOPS_PER_CELL = 1332
STEP_FLOPS_PER_CELL = 5060


def fusion_bytes(kernel, w, elt):
    """Bytes per step a kernel moves beyond the method's own words because of a
    fusion choice: the stress kernel writes the summed stress tau^k + tau^{k-1}
    (6 words per substep) that the momentum kernel then reads instead of B^{k-1}
    and B^k (12 words)."""
    N = w['nx'] * w['ny'] * w['nz']
    return 3 * 6 * N * elt if kernel == 'stress_weno_update' else 0


# CUDA sources that determine each profiled kernel's code (for the staleness check)
KERNEL_SOURCES = {
    'stress_weno_update': ['k_stress.cuh', 'k_stress_f32.cu', 'weno.cuh', 'evp_internal.cuh'],
}


def kernel_sources_sha256(kernel):
    """SHA-256 over the CUDA sources of ``kernel`` (file names and contents, in order)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        h.update(f.encode())
        with open(os.path.join(ROOT, 'paper_1803_09563_gb300', 'csrc', f), 'rb') as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary of this kernel, or None
    when there is none or its kernel sources have changed since it was captured."""
    p = os.path.join(ROOT, 'profiles', f'{kernel}__channel_256x128x128_fp32.md')
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    traffic, sha = None, None
    for line in open(p):
        if line.startswith('traffic_bytes_per_launch:'):
            try:
                traffic = float(line.split(':', 1)[1])
            except ValueError:
                return None
        elif line.startswith('source_sha256:'):
            sha = line.split(':', 1)[1].strip()
    return traffic if sha == kernel_sources_sha256(kernel) else None


def max_over_ranks(x, world, device):
    """Max of a scalar over all ranks (the slowest replica sets the job time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells, steps, world, seconds):
    """Whole-job Mcell-steps/s: every replica advances ``cells`` for ``steps`` steps."""
    return cells * steps * world / seconds / 1e6


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1803_09563_gb300 import evp
    torch.cuda.set_device(local_rank)
    w = WORKLOAD
    N = w['nx'] * w['ny'] * w['nz']
    geo, U, V, W = workload_inputs(w)
    stream = torch.cuda.Stream()

    def make(precision):
        grid = evp.make_grid(w['nx'], w['ny'], w['nz'], w['lx'], w['ly'], w['lz'], w['walls_y'])
        prm = evp.make_params(Re=w['Re'], Wi=w['Wi'], beta=w['beta'], Bi=w['Bi'], dpdx=2.0 / w['Re'],
                              precision=precision)
        sim = evp.Simulation(grid, w['model'], prm, stream=stream.cuda_stream)
        sim.set_state(U, V, W)
        return sim

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_ranks(x):
        return max_over_ranks(x, world, 'cuda')

    # ---------------- FP32-served: timed region (CUDA-graph replay of each step, the
    # library's production path; no per-kernel instrumentation inside it)
    sim = make(evp.EVP_FP32)
    evp.evp_set_graph(sim.handle, True)
    for _ in range(args.warmup):
        sim.step(w['dt'])
    sim.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    clocks.wait_first()
    barrier()
    torch.cuda.synchronize()
    clocks.begin()
    ev[0].record(stream)
    for k in range(args.steps):
        sim.step(w['dt'])
        ev[k + 1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks.end()
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    code, bits, maxdiv = sim.sync(raise_on_error=False)
    total_ms = max_ranks(total_ms)
    value = job_rate(N, args.steps, world, total_ms * 1e-3)
    # per-kernel durations: an adjacent pass over the same workload with a CUDA event
    # pair around every launch on the library stream (direct launches: events cannot
    # sit between the kernels of a replayed graph)
    k_steps = max(10, min(args.steps, 40))
    evp.evp_kernel_timing(sim.handle, True)
    evp.evp_kernel_times(sim.handle)       # reset counters
    for _ in range(k_steps):
        sim.step(w['dt'])
    ktimes = evp.evp_kernel_times(sim.handle)
    evp.evp_kernel_timing(sim.handle, False)
    per_step_launches = sum(c for _, c in ktimes.values()) / k_steps
    launches = int(round(per_step_launches * args.steps))

    # roofline of the dominant kernel (largest share of device time)
    hbm, peak_kind = peaks()
    elt = 4
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    kern = {}
    for name, (ms, cnt) in ktimes.items():
        if cnt == 0:
            continue
        b, per = algorithmic_bytes(name, w, elt, w['walls_y'])
        nsteps = cnt / per
        gbs = b * nsteps / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        kern[name] = {"ms_per_launch": ms / cnt, "launches": cnt, "share": ms / sum(v[0] for v in ktimes.values()),
                      "algorithmic_GBps": gbs, "frac_of_hbm": gbs / hbm}
        fb = fusion_bytes(name, w, elt)
        if fb:
            # bytes the kernel moves beyond the method's own (the summed stress it writes)
            kern[name]["fusion_GBps"] = fb * nsteps / (ms * 1e-3) / 1e9
            kern[name]["with_fusion_frac_of_hbm"] = (b + fb) * nsteps / (ms * 1e-3) / 1e9 / hbm
    b_dom, per_dom = algorithmic_bytes(dom, w, elt, w['walls_y'])
    dom_ms, dom_cnt = ktimes[dom]
    achieved = b_dom * (dom_cnt / per_dom) / (dom_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom)

    # plain-FMA peaks of this GPU (non-tensor FP32 and FP64), the arithmetic roofline
    fma = {"fp32_tflops": evp.evp_fma_peak(evp.EVP_FP32) / 1e12, "fp64_tflops": evp.evp_fma_peak(evp.EVP_FP64) / 1e12,
           "how": "evp_fma_peak: 8 independent FMA chains per thread, 8 blocks of 256 threads per SM, "
                  "packed f32x2 FMAs in FP32; best of 3 timed launches, an FMA counted as 2 operations"}

    # ---------------- e2e through the C ABI with host buffers: replicas of the
    # state, each on its own stream, stepping in turn with evp_step_io: every step
    # copies its 10 fields in from pinned host memory, takes one RK3 step and copies
    # the 10 fields back out to the same host buffers (the state makes the round
    # trip through host memory every step); one replica's copies overlap another's
    # step, nothing is waited for until the end
    fields_io = [evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P] + [evp.EVP_BXX + c for c in range(6)]
    host_a = [torch.empty(sim.shape, dtype=torch.float32).pin_memory() for _ in fields_io]
    for f, h in zip(fields_io, host_a):
        evp.evp_get_field(sim.handle, f, h.numpy())
    # further replicas start from the same state, each on its own stream
    NREP = 4
    pair = [sim]
    host = [host_a]
    grid_w = evp.make_grid(w['nx'], w['ny'], w['nz'], w['lx'], w['ly'], w['lz'], w['walls_y'])
    prm_w = evp.make_params(Re=w['Re'], Wi=w['Wi'], beta=w['beta'], Bi=w['Bi'], dpdx=2.0 / w['Re'],
                            precision=evp.EVP_FP32)
    rep_streams = []
    for _ in range(NREP - 1):
        hb = [h.clone().pin_memory() for h in host_a]
        st_r = torch.cuda.Stream()
        rep_streams.append(st_r)
        sr = evp.Simulation(grid_w, w['model'], prm_w, stream=st_r.cuda_stream)
        evp.evp_set_graph(sr.handle, True)
        for _ in range(2):               # capture the replica's graphs (both parities)
            sr.step(w['dt'])
        evp.evp_set_fields(sr.handle, fields_io, [h.numpy() for h in hb])
        pair.append(sr)
        host.append(hb)
    io = [evp.StepIO(fields_io, [h.numpy() for h in hb], fields_io, [h.numpy() for h in hb]) for hb in host]
    e2e_steps = NREP * max(1, args.steps // (2 * NREP))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        evp.evp_step_io(pair[k % NREP].handle, w['dt'], io[k % NREP])
    torch.cuda.synchronize()
    e2e_s = max_ranks(time.perf_counter() - t0)
    e2e_value = job_rate(N, e2e_steps, world, e2e_s)
    # the same calls on one replica: its copies and steps follow each other on its
    # stream, with nothing to overlap them (what the replicas buy)
    one_steps = max(8, e2e_steps // 8)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(one_steps):
        evp.evp_step_io(pair[0].handle, w['dt'], io[0])
    torch.cuda.synchronize()
    one_value = job_rate(N, one_steps, world, max_ranks(time.perf_counter() - t0))
    io_bytes = len(fields_io) * N * 4
    fp32_fields = [sim.get(f) for f in fields_io]
    for sr in pair:
        sr.close()

    # ---------------- FP64 plain on the same workload and the same steps
    sim64 = make(evp.EVP_FP64)
    n64 = max(2, args.steps // 4)
    for _ in range(min(args.warmup, 2)):
        sim64.step(w['dt'])
    sim64.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(n64):
        sim64.step(w['dt'])
    e1.record(stream)
    stream.synchronize()
    ms64 = max_ranks(e0.elapsed_time(e1))
    value64 = job_rate(N, n64, world, ms64 * 1e-3)
    # accuracy of FP32-served against FP64 plain after the same number of steps
    steps_done = args.warmup + args.steps + k_steps + e2e_steps // NREP + one_steps
    sim64.close()
    sim64 = make(evp.EVP_FP64)
    for _ in range(steps_done):
        sim64.step(w['dt'])
    sim64.sync()
    errs = {}
    for f, a in zip(fields_io, fp32_fields):
        b = sim64.get(f)
        errs[str(f)] = float(np.abs(a.astype(np.float64) - b).max() / max(np.abs(b).max(), 1e-300))
    sim64.close()

    sl = sorted(step_ms)
    p50 = sl[len(sl) // 2]
    p99 = sl[min(len(sl) - 1, int(round(0.99 * (len(sl) - 1))))]
    names = {evp.EVP_U: 'u', evp.EVP_V: 'v', evp.EVP_W: 'w', evp.EVP_P: 'p'}
    names.update({evp.EVP_BXX + c: 'B' + s for c, s in enumerate(['xx', 'xy', 'xz', 'yy', 'yz', 'zz'])})
    line = {
        "metric": METRIC, "value": value, "unit": "Mcell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (double-single Thomas sweep; FP64 divergence residual of the final state at sync)",
        "data": "synthetic (seeded Poiseuille + solenoidal perturbation)",
        "config": {"workload": w['name'], "grid": [w['nx'], w['ny'], w['nz']], "model": w['model'],
                   "Re": w['Re'], "Wi": w['Wi'], "Bi": w['Bi'], "beta": w['beta'], "dt": w['dt'],
                   "walls_y": True, "integrator": "RK3", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (state 0.66 GB per replica vs 129 MB L2)"},
        "p50_ms": p50, "p99_ms": p99,
        "fp64_plain": {"value": value64, "unit": "Mcell-steps/s", "steps": n64, "ms_per_step": ms64 / n64},
        "fp32_vs_fp64_rel_err": {names[int(k)]: v for k, v in errs.items()},
        "fp32_vs_fp64_after_steps": steps_done,
        "max_div_fp64_residual": maxdiv, "status_bits": bits,
        "e2e": {"value": e2e_value, "unit": "Mcell-steps/s", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes, "steps": e2e_steps,
                "how": f"evp_step_io: {NREP} replicas of the state on their own streams step in turn; each step "
                       "copies its 10 fields in from pinned host memory, takes one RK3 step and copies them back "
                       "out, so one replica's copies overlap another's step; host-clock time from the first call "
                       "to the final synchronisation",
                "one_replica": {"value": one_value, "steps": one_steps,
                                "how": "the same evp_step_io calls on one replica: copies in, step and copies out "
                                       "follow each other on its stream"}},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                     "traffic": traffic},
        "kernels": kern,
        "fma_peaks": fma,
        "alu_roofline": {
            "stress_weno_update": {"bound": "alu", "flops_per_cell": STRESS_FLOPS_PER_CELL,
                                   "achieved": STRESS_FLOPS_PER_CELL * N / (kern['stress_weno_update']['ms_per_launch'] * 1e-3) / 1e12,
                                   "peak": fma["fp32_tflops"], "unit": "TFLOP/s",
                                   "frac": STRESS_FLOPS_PER_CELL * N / (kern['stress_weno_update']['ms_per_launch'] * 1e-3) / 1e12 / fma["fp32_tflops"],
                                   "peak_kind": "measured FP32 FMA (evp_fma_peak)"}
            if 'stress_weno_update' in kern else None,
            "fp64_plain_step": {"bound": "alu", "flops_per_cell_step": STEP_FLOPS_PER_CELL,
                                "achieved": STEP_FLOPS_PER_CELL * value64 * 1e6 / world / 1e12,
                                "peak": fma["fp64_tflops"], "unit": "TFLOP/s",
                                "frac": STEP_FLOPS_PER_CELL * value64 * 1e6 / world / 1e12 / fma["fp64_tflops"],
                                "peak_kind": "measured FP64 FMA (evp_fma_peak)"},
            "note": "operation counts from the method's formulas (FMA = 2), not from the instructions executed"},
        "cufft_reference": cufft_reference(ktimes),
        "kernel_timing": f"adjacent pass of {k_steps} steps with CUDA events around each launch on the library "
                         f"stream (direct launches); the timed region replays a CUDA graph per step",
        "clocks": clk,
    }
    return line


def cufft_reference(ktimes):
    """cuFFT (through torch.fft), timed as a reference point only, on the transforms
    the hand-written passes of the channel's Poisson solve take: the real-to-complex
    transform along x of a 128 x 128 x 256 FP32 field, the complex transform along
    z of its (129-wide) spectrum, and the two inverses; beside it the hand-written
    chain's x and z passes (div_fft_x + fft_z_forward + fft_z_inverse + ifft_x_psi,
    per substep, from the instrumented pass).  Also the 256^3 FP32 periodic
    real-to-complex 3-D transform pair (rfftn + irfftn) of the FENE-P box."""
    import torch
    out = {}
    x = torch.randn(128, 128, 256, device='cuda', dtype=torch.float32)

    def timeit(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    def chain():
        X = torch.fft.rfft(x, dim=2)
        X = torch.fft.fft(X, dim=0)
        X = torch.fft.ifft(X, dim=0)
        return torch.fft.irfft(X, n=256, dim=2)
    out["channel_x_z_transforms_ms"] = timeit(chain)
    mine = 0.0
    for k in ('div_fft_x', 'fft_z_forward', 'fft_z_inverse', 'ifft_x_psi'):
        ms, cnt = ktimes.get(k, (0.0, 0))
        if cnt:
            mine += ms / cnt
    out["hand_written_x_z_passes_ms"] = mine
    del x
    y = torch.randn(256, 256, 256, device='cuda', dtype=torch.float32)
    out["periodic_256^3_rfftn_irfftn_ms"] = timeit(lambda: torch.fft.irfftn(torch.fft.rfftn(y), s=y.shape), reps=10)
    out["note"] = ("cuFFT is a reference point only: the hand-written passes also fuse the divergence into the "
                   "x pass and the scaling into the inverse x pass")
    del y
    torch.cuda.empty_cache()
    return out


def run_serving(requests=64):
    """Serving mix: a seeded Poisson stream (0.05 requests per ms, seed 3) of 64
    periodic Saramito requests, grids from {32, 48, 64, 96, 128}^3, Wi in U[0.5, 4],
    Bi in U[0, 1], beta in U[0.3, 0.9], random solenoidal velocity (|k| <= 4,
    max-norm 1), 100-1000 FP32 steps each, admitted under a 120 GB budget; one
    batch per grid size, its tiles autotuned before the run (untimed)."""
    from paper_1803_09563_gb300 import serve
    reqs = serve.mixed_requests(64, seed=3, steps=(100, 1000), rate_per_ms=0.05)[:requests]
    prepared = {r.rid: serve.request_inputs(r) for r in reqs}      # client side, untimed
    srv = serve.Server(budget_bytes=120 * 10 ** 9, result_fields=(), tune=False)
    t0 = time.perf_counter()
    tuned = srv.tune_sizes(reqs)
    tune_s = time.perf_counter() - t0
    _, rep = srv.run(reqs, prepared=prepared)
    rep["tuned_tiles"] = {str(n): {"config": list(c), "ms_per_step": ms} for n, (c, ms) in tuned.items()}
    rep["tune_seconds"] = tune_s
    rep["steps_per_request"] = [100, 1000]
    rep["workload"] = "serving_mix_64_requests_32-128^3_saramito_fp32_100-1000_steps_120GB"
    return rep


def run_fene_turbulence(steps=4):
    """FENE-P forced turbulence: triply periodic 256^3 on a 2 pi box, L^2 = 900,
    Wi = 5, beta = 0.9, Re = 200, ABC forcing (A = 1, k = 2), initial solenoidal
    velocity with a k^-5/3 spectrum for 1 <= |k| <= 16 (u_rms = 1, seed 2), B = I,
    dt = 1e-3.  FP32 and FP64 side by side from the same state; the relative
    difference of every field after ``steps`` steps is reported."""
    import torch
    from paper_1803_09563_gb300 import evp, inputs
    n, L = 256, 2 * np.pi
    geo = inputs.geometry(n, n, n, L, L, L)
    U, V, W = inputs.scale_rms(*inputs.random_solenoidal(geo, 2, 16, spectrum='k-5/3', periodic_fft=True), 1.0)
    out = {"workload": "fene_p_turbulence_256^3", "steps": steps}
    res = {}
    for prec, name in ((evp.EVP_FP32, 'fp32'), (evp.EVP_FP64, 'fp64')):
        stream = torch.cuda.Stream()
        sim = evp.Simulation(evp.make_grid(n, n, n, L, L, L), 'fene_p',
                             evp.make_params(Re=200.0, Wi=5.0, beta=0.9, L2=900.0, abc_amp=1.0, abc_k=2.0,
                                             precision=prec), stream=stream.cuda_stream)
        sim.set_state(U, V, W)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sim.step(1e-3)
        sim.sync()
        e0.record(stream)
        for _ in range(steps - 1):
            sim.step(1e-3)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / max(1, steps - 1)
        code, bits, maxdiv = sim.sync(raise_on_error=False)
        out[name] = {"ms_per_step": ms, "Mcell_steps_per_s": n ** 3 / (ms * 1e-3) / 1e6, "max_div": maxdiv,
                     "status": code}
        res[name] = [sim.get(f).astype(np.float64) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_BXX,
                                                                 evp.EVP_BXY)]
        if name == 'fp32':
            # per-kernel times of one more, instrumented step (after the fields were
            # read): the periodic Poisson chain beside cuFFT's 3-D transform pair
            evp.evp_kernel_timing(sim.handle, True)
            evp.evp_kernel_times(sim.handle)
            sim.step(1e-3)
            kt = evp.evp_kernel_times(sim.handle)
            evp.evp_kernel_timing(sim.handle, False)
            out[name]["kernels_ms_per_launch"] = {k: t / c for k, (t, c) in kt.items() if c}
            out[name]["hand_written_periodic_chain_ms"] = sum(
                kt[k][0] / kt[k][1] for k in ('div_fft_x', 'fft_z_forward', 'fft_y_modal_solve', 'fft_z_inverse',
                                              'ifft_x_psi') if kt.get(k, (0, 0))[1])
        sim.close()
    out["fp32_vs_fp64_rel_err"] = {k: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
                                   for k, a, b in zip(('u', 'v', 'w', 'Bxx', 'Bxy'), res['fp32'], res['fp64'])}
    return out


def run_evp_drop(steps=20):
    """Two-phase buoyancy-driven drop in a Saramito EVP fluid: 128 x 256 x 128, triply
    periodic 4 x 8 x 4 box, FP32, AB2 with the level set.  Drop of radius 0.5 centred
    at (2, 2, 2) from rest, Heaviside smoothed over 1.5 cells, Boussinesq buoyancy with
    drho g = 1 and surface tension 0.1 (Bond = drho g D^2 / sigma = 10), Re = 10,
    Wi = 1, Bi = 0.2 (tau_y = Bi), beta = 0.5, viscosity ratio 1, re-distancing (two
    pseudo-steps) every 10 steps, dt = 1e-3.  Reports the step rate and the per-kernel
    split of an adjacent pass with event timing; the level-set kernel's algorithmic
    bytes are 6 words per cell for an advection stage (u, v, w, phi^n, stage input
    read, phi written) and 4 for a re-distancing stage (phi0 instead of u, v, w)."""
    import torch
    from paper_1803_09563_gb300 import evp, inputs
    nx, ny, nz = 128, 256, 128
    N = nx * ny * nz
    geo = inputs.geometry(nx, ny, nz, 4.0, 8.0, 4.0)
    phi = inputs.sphere_distance(geo, (2.0, 2.0, 2.0), 0.5)
    prm = evp.make_params(Re=10.0, Wi=1.0, beta=0.5, Bi=0.2, bi_def=1, precision=evp.EVP_FP32,
                          integrator=evp.EVP_AB2, mu_ratio=1.0, ls_eps_cells=1.5, sigma=0.1, drho_g=1.0,
                          reinit_every=10, reinit_iters=2)
    stream = torch.cuda.Stream()
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, 4.0, 8.0, 4.0), 'saramito', prm, stream=stream.cuda_stream)
    sim.set(evp.EVP_PHI, phi)
    dt = 1e-3
    for _ in range(3):
        sim.step(dt)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.step(dt)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    k_steps = 10
    evp.evp_kernel_timing(sim.handle, True)
    evp.evp_kernel_times(sim.handle)
    for _ in range(k_steps):
        sim.step(dt)
    kt = evp.evp_kernel_times(sim.handle)
    evp.evp_kernel_timing(sim.handle, False)
    code, bits, maxdiv = sim.sync(raise_on_error=False)
    sim.close()
    total = sum(t for t, c in kt.values() if c)
    kern = {k: {"ms_per_launch": t / c, "launches_per_step": c / k_steps, "share": t / total}
            for k, (t, c) in kt.items() if c}
    out = {"workload": "evp_drop_128x256x128_fp32_ab2", "steps": steps, "ms_per_step": ms,
           "Mcell_steps_per_s": N / (ms * 1e-3) / 1e6, "max_div": maxdiv, "status": code, "kernels": kern}
    ls_ms, ls_n = kt.get('levelset_stage', (0.0, 0))
    if ls_n:
        n_adv = 3 * k_steps
        ls_bytes = N * 4 * (6 * n_adv + 4 * (ls_n - n_adv))
        gbs = ls_bytes / (ls_ms * 1e-3) / 1e9
        hbm, _ = peaks()
        out["levelset_stage_algorithmic_GBps"] = gbs
        out["levelset_stage_frac_of_hbm"] = gbs / hbm
    return out


def run_implicit_viscous(steps=50):
    """The C2 channel with the implicit viscous option (three Helmholtz solves per
    substep), FP32, graph replay: what the literal reading of Eq. NS-num1 costs."""
    import torch
    from paper_1803_09563_gb300 import evp
    w = WORKLOAD
    geo, U, V, W = workload_inputs(w)
    stream = torch.cuda.Stream()
    out = {"workload": "saramito_channel_256x128x128_fp32_implicit_viscous", "steps": steps}
    for name, vi in (('explicit', 0), ('implicit', 1)):
        grid = evp.make_grid(w['nx'], w['ny'], w['nz'], w['lx'], w['ly'], w['lz'], w['walls_y'])
        prm = evp.make_params(Re=w['Re'], Wi=w['Wi'], beta=w['beta'], Bi=w['Bi'], dpdx=2.0 / w['Re'],
                              precision=evp.EVP_FP32, viscous_implicit=vi)
        sim = evp.Simulation(grid, w['model'], prm, stream=stream.cuda_stream)
        sim.set_state(U, V, W)
        evp.evp_set_graph(sim.handle, True)
        for _ in range(3):
            sim.step(w['dt'])
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sim.step(w['dt'])
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "Mcell_steps_per_s": w['nx'] * w['ny'] * w['nz'] / (ms * 1e-3) / 1e6}
        sim.close()
    return out


def run_thomas_sweeps(steps=200):
    """The C2 channel in FP32 with the wall-normal Thomas sweep in double-single
    arithmetic (the default) and in FP64 (thomas_fp64 = 1): step time and the
    sweep's own time, and the largest difference between the two runs' fields."""
    import torch
    from paper_1803_09563_gb300 import evp
    w = WORKLOAD
    geo, U, V, W = workload_inputs(w)
    stream = torch.cuda.Stream()
    out = {"workload": "saramito_channel_256x128x128_fp32", "steps": steps}
    fields = {}
    for name, t in (('double_single', 0), ('fp64', 1)):
        grid = evp.make_grid(w['nx'], w['ny'], w['nz'], w['lx'], w['ly'], w['lz'], w['walls_y'])
        prm = evp.make_params(Re=w['Re'], Wi=w['Wi'], beta=w['beta'], Bi=w['Bi'], dpdx=2.0 / w['Re'],
                              precision=evp.EVP_FP32, thomas_fp64=t)
        sim = evp.Simulation(grid, w['model'], prm, stream=stream.cuda_stream)
        sim.set_state(U, V, W)
        evp.evp_set_graph(sim.handle, True)
        for _ in range(3):
            sim.step(w['dt'])
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sim.step(w['dt'])
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # the sweep's own time: an instrumented pass of direct launches
        evp.evp_kernel_timing(sim.handle, True)
        evp.evp_kernel_times(sim.handle)
        for _ in range(5):
            sim.step(w['dt'])
        kt = evp.evp_kernel_times(sim.handle)
        evp.evp_kernel_timing(sim.handle, False)
        t_ms, n = kt['thomas_y']
        out[name] = {"ms_per_step": ms, "Mcell_steps_per_s": w['nx'] * w['ny'] * w['nz'] / (ms * 1e-3) / 1e6,
                     "thomas_us_per_launch": 1e3 * t_ms / max(n, 1)}
        fields[name] = [sim.get(f) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_BXX, evp.EVP_BXY)]
        sim.close()
    rel = 0.0
    for a, b in zip(fields['double_single'], fields['fp64']):
        a = a.astype(np.float64)
        b = b.astype(np.float64)
        rel = max(rel, float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)))
    out["max_rel_diff_u_v_w_Bxx_Bxy"] = rel
    out["steps_compared"] = 3 + steps + 5
    return out


def run_small_grid():
    """Single-phase Oldroyd-B Taylor-Green box 32^3 in FP64 (the 10-step parity
    workload): per-step latency with direct launches and with graph replay."""
    import torch
    from paper_1803_09563_gb300 import evp, inputs
    n, L = 32, 2 * np.pi
    geo = inputs.geometry(n, n, n, L, L, L)
    U, V, W = inputs.taylor_green(geo)
    out = {}
    for graph in (False, True):
        stream = torch.cuda.Stream()
        sim = evp.Simulation(evp.make_grid(n, n, n, L, L, L), 'oldroyd_b',
                             evp.make_params(Re=1.0, Wi=1.0, beta=0.5, precision=evp.EVP_FP64),
                             stream=stream.cuda_stream)
        sim.set_state(U, V, W)
        if graph:
            evp.evp_set_graph(sim.handle, True)
        for _ in range(4):
            sim.step(1e-3)
        sim.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = 200
        e0.record(stream)
        for _ in range(steps):
            sim.step(1e-3)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["graph" if graph else "direct"] = {"ms_per_step": ms, "Mcell_steps_per_s": n ** 3 / (ms * 1e-3) / 1e6}
        sim.close()
    out["workload"] = "oldroyd_b_taylor_green_32^3_fp64"
    return out


def _oracle_slab(nz):
    """Oracle state of a 256 x 128 x nz slab of the channel (inputs only)."""
    import oracle
    w = WORKLOAD
    geo, U, V, W = workload_inputs(w, nz=nz)
    g = oracle.Grid(w['nx'], w['ny'], nz, geo['lx'], geo['ly'], geo['lz'], True)
    prm = oracle.Params.from_groups(w['model'], w['Re'], w['Wi'], w['beta'], Bi=w['Bi'])
    return g, prm, oracle.State.rest(g, U, V, W)


def _oracle_step(g, prm, s):
    import oracle
    w = WORKLOAD
    return oracle.rk3_step(s, w['dt'], g, prm, (2.0 / w['Re'], 0.0, 0.0))


def _oracle_worker(nz, barrier, queue):
    """One host process of the all-core run: build its slab, wait for the others,
    time one RK3 step of the oracle."""
    os.environ.setdefault('OMP_NUM_THREADS', '1')
    g, prm, s = _oracle_slab(nz)
    barrier.wait()
    t0 = time.time()
    _oracle_step(g, prm, s)
    queue.put((t0, time.time(), g.ncells))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_cpu_baseline(args, all_cores=True):
    """The FP64 oracle, as it stands, on bounded samples of the same workload.
    Single core: one RK3 step of a 256 x 128 x 64 slab of the channel (z halved).
    All cores: one process per host core (spawned, so no process is forked from a
    CUDA context), each timing one RK3 step of its own 256 x 128 x 32 slab after a
    barrier; throughput = all slabs' cells / (last end - first start)."""
    nz = 64
    g, prm, s = _oracle_slab(nz)
    t0 = time.perf_counter()
    _oracle_step(g, prm, s)
    dt = time.perf_counter() - t0
    single = {"value": g.ncells / dt / 1e6, "unit": "Mcell-steps/s", "cores": 1, "kind": "oracle",
              "sample": f"1 RK3 step of a {g.nx}x{g.ny}x{nz} slab of the channel (numpy FP64, "
                        f"single thread), {dt:.1f} s"}
    del s
    if not all_cores:
        return single
    import multiprocessing as mp
    n = host_cores()
    ctx = mp.get_context('spawn')
    barrier, queue = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(32, barrier, queue)) for _ in range(n)]
    for p in procs:
        p.start()
    res = [queue.get(timeout=600) for _ in range(n)]
    for p in procs:
        p.join(timeout=60)
    wall = max(r[1] for r in res) - min(r[0] for r in res)
    cells = sum(r[2] for r in res)
    return {"value": cells / wall / 1e6, "unit": "Mcell-steps/s", "cores": n, "kind": "oracle",
            "sample": f"{n} processes (one per host core), each one RK3 step of its own 256x128x32 slab of "
                      f"the channel (numpy FP64), {wall:.1f} s from the first start to the last end",
            "single_core": single}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=1600)
    ap.add_argument('--warmup', type=int, default=5)
    ap.add_argument('--impl', default='gpu', choices=['gpu', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-extras', action='store_true', help='skip the serving-mix and small-grid sections')
    ap.add_argument('--profile-case', default=None,
                    help='profiling runs only: "channel-nz=<n>" (the channel workload with n z planes, no '
                         'extras) or "serving=<n>" (the first n requests of the serving mix alone); prints the '
                         'section\'s JSON')
    args = ap.parse_args()
    rank = int(os.environ.get('RANK', 0))
    world = int(os.environ.get('WORLD_SIZE', 1))
    local_rank = int(os.environ.get('LOCAL_RANK', 0))

    if args.impl == 'reference':
        # the oracle is the reference arm: rank 0 only, host cores, bounded samples
        if rank != 0:
            return
        # untimed warm-up samples, then the timed ones; both capped at 3 so that the
        # run stays within a few minutes of host time
        warm = max(0, min(args.warmup, 2))
        for _ in range(warm):
            run_cpu_baseline(args)
        vals = []
        for _ in range(max(1, min(args.steps, 3))):
            vals.append(run_cpu_baseline(args))
        v = statistics.median(x['value'] for x in vals)
        cb = dict(vals[0])
        cb['value'] = v
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mcell-steps/s", "n_gpus": world,
                "steps": len(vals), "warmup": warm, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD['name']}, "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "Mcell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.profile_case:
        # smaller cases for ncu captures (not bench lines)
        kind, _, n = args.profile_case.partition('=')
        if kind == 'serving':
            print(json.dumps({"profile_case": args.profile_case, "serving": run_serving(requests=int(n))}))
        elif kind == 'channel-nz':
            WORKLOAD['nz'] = int(n)
            WORKLOAD['lz'] = 2 * np.pi * int(n) / 128
            WORKLOAD['name'] = f"saramito_channel_256x128x{int(n)}"
            line = run_gpu(args, 0, 1, 0)
            print(json.dumps({"profile_case": args.profile_case, "kernels": line['kernels']}))
        else:
            raise SystemExit(f'unknown profile case {args.profile_case}')
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group('nccl', device_id=torch.device('cuda', local_rank))
    line = run_gpu(args, rank, world, local_rank)
    if not args.no_extras:
        line['serving'] = run_serving()
        line['small_grid'] = run_small_grid()
        line['fene_p_turbulence'] = run_fene_turbulence()
        line['implicit_viscous'] = run_implicit_viscous()
        line['thomas_sweeps'] = run_thomas_sweeps()
        line['evp_drop'] = run_evp_drop()
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line['cpu_baseline'] = run_cpu_baseline(args)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
