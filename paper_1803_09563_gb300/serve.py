"""Continuous batching of EVP simulations on one GPU.

Requests (grid size, Wi / Bi / beta, number of steps, seed) arrive over time.
The server keeps every admitted simulation resident on the device and groups the
residents by grid size into classes; each class is one libevp batch
(``evp_batch_*``) on its own CUDA stream, so one replayed CUDA graph advances all
of a class's members by one step with one launch per kernel phase, and classes of
different sizes overlap on the device.

The host loop never waits for the device: it polls each class's end-of-step
event (``cudaEventQuery``).  When a class's step has finished, its finished
members are evicted (result read back, arena freed), waiting requests of that
size are admitted while the HBM budget (``evp_state_bytes``) allows, and the
class's next step is launched at once.  A small request therefore waits for
steps of its own size class only, never for the largest grid resident.

Reported per request-step: the step latency (device time from the start to the
end of the class step that advanced it, CUDA events) and, per request, the
queueing delay from its arrival to its admission (host clock).  Throughput is
cell-steps over the whole run.  Each result carries the final state's status,
FP64 divergence residual and monitoring quantities (evp_diagnostics: kinetic
energy, det B and tr B extremes, yielded fraction, non-finite cells) beside the
requested fields.

The loop is host logic only: every step of every simulation runs in libevp's
kernels through the C ABI.
"""

import time
from dataclasses import dataclass, field

import numpy as np

from . import evp, inputs


@dataclass(order=True)
class Request:
    arrival_ms: float
    rid: int
    n: int = field(compare=False)
    Wi: float = field(compare=False)
    Bi: float = field(compare=False)
    beta: float = field(compare=False)
    steps: int = field(compare=False)
    seed: int = field(compare=False)
    Re: float = field(default=100.0, compare=False)
    dt: float = field(default=1e-3, compare=False)


def mixed_requests(count, seed, grids=(32, 48, 64, 96, 128), steps=(100, 1000), rate_per_ms=1.0):
    """A seeded Poisson stream of periodic Saramito requests (grid drawn from
    ``grids``, Wi in U[0.5, 4], Bi in U[0, 1], beta in U[0.3, 0.9], step counts in
    U[steps]) arriving at ``rate_per_ms`` requests per millisecond on average."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_per_ms)
        out.append(Request(arrival_ms=float(t), rid=rid, n=int(rng.choice(grids)), Wi=float(rng.uniform(0.5, 4.0)),
                           Bi=float(rng.uniform(0.0, 1.0)), beta=float(rng.uniform(0.3, 0.9)),
                           steps=int(rng.integers(steps[0], steps[1] + 1)), seed=int(rng.integers(1 << 30))))
    return out


def request_inputs(req):
    """Random solenoidal velocity, |k| <= 4, max-norm 1, on a 2 pi periodic box."""
    L = 2 * np.pi
    geo = inputs.geometry(req.n, req.n, req.n, L, L, L)
    return inputs.scale_max(*inputs.random_solenoidal(geo, req.seed, 4), 1.0)


def request_grid(req):
    L = 2 * np.pi
    return evp.make_grid(req.n, req.n, req.n, L, L, L)


def request_params(req, precision):
    return evp.make_params(Re=req.Re, Wi=req.Wi, beta=req.beta, Bi=req.Bi, precision=precision)


class Instance:
    """One admitted request: its libevp state with the request's initial velocity."""

    def __init__(self, req, precision, fields=None):
        self.req = req
        self.grid = request_grid(req)
        self.params = request_params(req, precision)
        self.bytes = evp.evp_state_bytes(self.grid, evp.EVP_SARAMITO, self.params)
        self.sim = evp.Simulation(self.grid, 'saramito', self.params)
        U, V, W = fields if fields is not None else request_inputs(req)
        self.sim.set_state(U, V, W)
        self.done = 0
        self.cells = req.n ** 3


class SizeClass:
    """The residents of one grid size: a libevp batch on its own stream."""

    def __init__(self, n, precision, use_graph):
        import torch
        self.n = n
        # small grids on a high-priority stream: their short steps get SMs as soon
        # as the large classes' CTAs retire
        self.stream = torch.cuda.Stream(priority=-1 if n <= 64 else 0)
        self.batch = evp.Batch(precision, stream=self.stream.cuda_stream)
        evp.evp_batch_set_graph(self.batch.handle, use_graph)
        self.members = []
        self.start = torch.cuda.Event(enable_timing=True)
        self.end = torch.cuda.Event(enable_timing=True)
        self.in_flight = False

    def launch(self):
        self.start.record(self.stream)
        self.batch.step()
        self.end.record(self.stream)
        self.in_flight = True

    def close(self):
        self.batch.close()


class Server:
    def __init__(self, budget_bytes, precision=evp.EVP_FP32, use_graph=True,
                 result_fields=(evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P, evp.EVP_BXY), tune=False):
        self.budget = int(budget_bytes)
        self.precision = precision
        self.use_graph = use_graph
        self.result_fields = result_fields
        self.tune = tune

    def tune_sizes(self, requests):
        """Autotune the batched kernels' tiles for every grid size of the stream
        (libevp's evp_tune, coordinate descent); returns {n: (config, ms/step)}."""
        out = {}
        for n in sorted({r.n for r in requests}):
            r = next(x for x in requests if x.n == n)
            cfg, ms, _ = evp.evp_tune(request_grid(r), 'saramito', request_params(r, self.precision))
            out[n] = (cfg.as_tuple(), ms)
        return out

    def run(self, requests, prepared=None, max_seconds=600.0):
        """Serve ``requests`` (arrival times in ms from the start of the run);
        returns (results by rid, report dict).  ``prepared`` maps rid -> (U, V, W)
        initial velocities generated by the client ahead of time (otherwise they
        are generated at admission)."""
        import torch
        tuned = self.tune_sizes(requests) if self.tune else None
        waiting = sorted(requests)
        ready = []              # arrived, not yet admitted (arrival order)
        classes = {}
        results = {}
        lat = []
        lat_by_n = {}
        queue_ms = []
        used = 0
        cell_steps = 0
        resident_hist = []
        max_resident = 0
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        wi = 0
        while wi < len(waiting) or ready or any(c.members for c in classes.values()):
            now = (time.perf_counter() - t_start) * 1e3
            if now > max_seconds * 1e3:
                raise RuntimeError('serving loop exceeded its time limit')
            while wi < len(waiting) and waiting[wi].arrival_ms <= now:
                ready.append(waiting[wi])
                wi += 1
            progressed = False
            # finished class steps: account, evict finished members
            for c in classes.values():
                if c.in_flight and c.end.query():
                    c.in_flight = False
                    progressed = True
                    dur = c.start.elapsed_time(c.end)
                    keep = []
                    for inst in c.members:
                        lat.append(dur)
                        lat_by_n.setdefault(c.n, []).append(dur)
                        inst.done += 1
                        cell_steps += inst.cells
                        if inst.done >= inst.req.steps:
                            c.batch.evict(inst.sim)
                            code, bits, maxdiv = inst.sim.sync(raise_on_error=False)
                            results[inst.req.rid] = dict(code=code, bits=bits, max_div=maxdiv,
                                                         diagnostics=inst.sim.diagnostics(),
                                                         fields={f: inst.sim.get(f) for f in self.result_fields})
                            inst.sim.close()
                            used -= inst.bytes
                        else:
                            keep.append(inst)
                    c.members = keep
            # admission: arrival order within each size class, into idle classes,
            # while the budget allows
            still = []
            for req in ready:
                c = classes.get(req.n)
                need = evp.evp_state_bytes(request_grid(req), evp.EVP_SARAMITO,
                                           request_params(req, self.precision))
                busy = c is not None and c.in_flight
                full = c is not None and len(c.members) >= evp.EVP_BATCH_MAX
                if busy or full or used + need > self.budget or any(r.n == req.n for r in still):
                    still.append(req)
                    continue
                if c is None:
                    c = classes[req.n] = SizeClass(req.n, self.precision, self.use_graph)
                inst = Instance(req, self.precision, None if prepared is None else prepared.get(req.rid))
                c.batch.admit(inst.sim, req.dt)
                c.members.append(inst)
                used += inst.bytes
                queue_ms.append((time.perf_counter() - t_start) * 1e3 - req.arrival_ms)
                progressed = True
            ready = still
            # launch the next step of every idle class with members
            nres = sum(len(c.members) for c in classes.values())
            for c in classes.values():
                if not c.in_flight and c.members:
                    c.launch()
                    resident_hist.append(nres)
                    progressed = True
            max_resident = max(max_resident, nres)
            if not progressed:
                time.sleep(20e-6)
        torch.cuda.synchronize()
        total_s = time.perf_counter() - t_start
        for c in classes.values():
            c.close()

        def pct(v, q):
            v = sorted(v)
            return v[min(len(v) - 1, int(round(q * (len(v) - 1))))] if v else None
        report = {
            "requests": len(results), "cell_steps": cell_steps, "request_steps": len(lat),
            "value": cell_steps / total_s / 1e6 if total_s > 0 else None, "unit": "Mcell-steps/s",
            "seconds": total_s,
            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
            "queue_p50_ms": pct(queue_ms, 0.5), "queue_p99_ms": pct(queue_ms, 0.99),
            "mean_resident": float(np.mean(resident_hist)) if resident_hist else 0.0,
            "max_resident": int(max_resident),
            "size_classes": sorted(classes),
            "by_size": {str(n): {"request_steps": len(v), "p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99)}
                        for n, v in sorted(lat_by_n.items())},
        }
        if tuned is not None:
            report["tuned_tiles"] = {str(n): {"config": list(cfg), "ms_per_step": ms} for n, (cfg, ms) in tuned.items()}
        return results, report
