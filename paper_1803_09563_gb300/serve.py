"""Continuous batching of EVP simulations on one GPU.

Requests (grid size, Wi / Bi / beta, number of steps, seed) arrive over time.
The server admits a waiting request as soon as its state fits in the HBM budget
(``evp_state_bytes``) and a slot is free, keeps every admitted simulation
resident on the device, and advances all of them one step per tick: each
simulation runs on its own CUDA stream with its RK3 step replayed from a CUDA
graph, so the steps of different simulations overlap on the device.  Finished
simulations are evicted (their result is read back and their arena freed) and
their slot and memory go to the next waiting request.

Per-step latency of a simulation is measured on the device from the start of
the tick to the end of that simulation's step (CUDA events); the report gives
p50/p99 over all simulation-steps and the throughput in Mcell-steps/s.

The loop is host logic only: every step of every simulation runs in libevp's
kernels through the C ABI.
"""

import heapq
from dataclasses import dataclass, field

import numpy as np

from . import evp, inputs


@dataclass(order=True)
class Request:
    arrival_tick: int
    rid: int
    n: int = field(compare=False)
    Wi: float = field(compare=False)
    Bi: float = field(compare=False)
    beta: float = field(compare=False)
    steps: int = field(compare=False)
    seed: int = field(compare=False)
    Re: float = field(default=100.0, compare=False)
    dt: float = field(default=1e-3, compare=False)


def mixed_requests(count, seed, grids=(32, 48, 64, 96, 128), steps=(100, 1000), rate=1.0):
    """A seeded Poisson stream of periodic Saramito requests (grid drawn from
    ``grids``, Wi in U[0.5, 4], Bi in U[0, 1], beta in U[0.3, 0.9], step counts in
    U[steps]) arriving at ``rate`` requests per tick on average."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        out.append(Request(arrival_tick=int(t), rid=rid, n=int(rng.choice(grids)), Wi=float(rng.uniform(0.5, 4.0)),
                           Bi=float(rng.uniform(0.0, 1.0)), beta=float(rng.uniform(0.3, 0.9)),
                           steps=int(rng.integers(steps[0], steps[1] + 1)), seed=int(rng.integers(1 << 30))))
    return out


def request_inputs(req):
    """Random solenoidal velocity, |k| <= 4, max-norm 1, on a 2 pi periodic box."""
    L = 2 * np.pi
    geo = inputs.geometry(req.n, req.n, req.n, L, L, L)
    return inputs.scale_max(*inputs.random_solenoidal(geo, req.seed, 4), 1.0)


class Instance:
    def __init__(self, req, precision, use_graph):
        import torch
        self.req = req
        self.stream = torch.cuda.Stream()
        L = 2 * np.pi
        self.grid = evp.make_grid(req.n, req.n, req.n, L, L, L)
        self.params = evp.make_params(Re=req.Re, Wi=req.Wi, beta=req.beta, Bi=req.Bi, precision=precision)
        self.bytes = evp.evp_state_bytes(self.grid, evp.EVP_SARAMITO, self.params)
        self.sim = evp.Simulation(self.grid, 'saramito', self.params, stream=self.stream.cuda_stream)
        U, V, W = request_inputs(req)
        self.sim.set_state(U, V, W)
        if use_graph:
            evp.evp_set_graph(self.sim.handle, True)
        self.done = 0
        self.cells = req.n ** 3


class Server:
    def __init__(self, budget_bytes, max_resident=64, precision=evp.EVP_FP32, use_graph=True,
                 result_fields=(evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P, evp.EVP_BXY)):
        self.budget = int(budget_bytes)
        self.max_resident = int(max_resident)
        self.precision = precision
        self.use_graph = use_graph
        self.result_fields = result_fields

    def run(self, requests, max_ticks=10 ** 9):
        """Serve ``requests``; returns (results by rid, report dict)."""
        import torch
        waiting = list(requests)
        heapq.heapify(waiting)
        ready = []            # arrived, not yet admitted (FIFO)
        resident = []
        results = {}
        lat = []
        used = 0
        cell_steps = 0
        resident_hist = []
        tick = 0
        tick_stream = torch.cuda.Stream()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(tick_stream)
        while (waiting or ready or resident) and tick < max_ticks:
            while waiting and waiting[0].arrival_tick <= tick:
                ready.append(heapq.heappop(waiting))
            # admission: first come, first served while memory and slots allow
            while ready and len(resident) < self.max_resident:
                req = ready[0]
                L = 2 * np.pi
                need = evp.evp_state_bytes(evp.make_grid(req.n, req.n, req.n, L, L, L), evp.EVP_SARAMITO,
                                           evp.make_params(Re=req.Re, Wi=req.Wi, beta=req.beta, Bi=req.Bi,
                                                           precision=self.precision))
                if used + need > self.budget:
                    break
                ready.pop(0)
                inst = Instance(req, self.precision, self.use_graph)
                used += inst.bytes
                resident.append(inst)
            if not resident:
                tick += 1
                continue
            resident_hist.append(len(resident))
            # one tick: every resident simulation advances one step on its own stream
            start = torch.cuda.Event(enable_timing=True)
            start.record(tick_stream)
            ends = []
            for inst in resident:
                inst.stream.wait_event(start)
                inst.sim.step(inst.req.dt)
                e = torch.cuda.Event(enable_timing=True)
                e.record(inst.stream)
                ends.append(e)
            for e in ends:
                e.synchronize()
            for inst, e in zip(resident, ends):
                lat.append(start.elapsed_time(e))
                inst.done += 1
                cell_steps += inst.cells
            # evict finished simulations
            keep = []
            for inst in resident:
                if inst.done >= inst.req.steps:
                    code, bits, maxdiv = inst.sim.sync(raise_on_error=False)
                    results[inst.req.rid] = dict(code=code, bits=bits, max_div=maxdiv,
                                                 fields={f: inst.sim.get(f) for f in self.result_fields})
                    inst.sim.close()
                    used -= inst.bytes
                else:
                    keep.append(inst)
            resident = keep
            tick += 1
        for e in (t1,):
            e.record(tick_stream)
        torch.cuda.synchronize()
        total_s = t0.elapsed_time(t1) * 1e-3
        lat_sorted = sorted(lat)
        report = {
            "requests": len(results), "ticks": tick, "cell_steps": cell_steps,
            "value": cell_steps / total_s / 1e6 if total_s > 0 else None, "unit": "Mcell-steps/s",
            "seconds": total_s,
            "p50_ms": lat_sorted[len(lat_sorted) // 2] if lat else None,
            "p99_ms": lat_sorted[min(len(lat_sorted) - 1, int(round(0.99 * (len(lat_sorted) - 1))))] if lat else None,
            "mean_resident": float(np.mean(resident_hist)) if resident_hist else 0.0,
            "max_resident": int(max(resident_hist)) if resident_hist else 0,
        }
        return results, report
