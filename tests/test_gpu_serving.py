"""Serving form: continuous batching of simulations of different sizes and
parameters (one libevp batch per grid size, stepped as its previous step ends).
Each request's result must be the same alone and in the mix (bitwise: every
member's arithmetic is its own), admission must respect the HBM budget, and
CUDA-graph replay must give the direct result."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def small_mix():
    from paper_1803_09563_gb300 import serve
    return serve.mixed_requests(8, seed=3, grids=(32, 48), steps=(4, 9), rate_per_ms=2.0)


def test_result_alone_equals_result_in_the_mix(evp):
    from paper_1803_09563_gb300 import serve
    reqs = small_mix()
    mixed, rep = serve.Server(budget_bytes=8 << 30).run(reqs)
    assert rep['requests'] == len(reqs) and rep['max_resident'] > 1
    for r in reqs:
        r0 = serve.Request(arrival_ms=0.0, rid=r.rid, n=r.n, Wi=r.Wi, Bi=r.Bi, beta=r.beta, steps=r.steps,
                           seed=r.seed)
        alone, _ = serve.Server(budget_bytes=8 << 30).run([r0])
        for f, a in alone[r.rid]['fields'].items():
            b = mixed[r.rid]['fields'][f]
            assert np.array_equal(a, b), (r.rid, f)
        assert mixed[r.rid]['code'] == 0
        # the monitoring quantities travel with the result, the same alone and in the mix
        d = mixed[r.rid]['diagnostics']
        assert d == alone[r.rid]['diagnostics']
        assert d['nonfinite_cells'] == 0 and d['min_det_B'] > 0 and 0.0 <= d['yielded_fraction'] <= 1.0
        U, V, W = (mixed[r.rid]['fields'][f].astype(np.float64) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W))
        dv = (2 * np.pi / r.n) ** 3
        assert d['kinetic_energy'] == pytest.approx(0.5 * dv * (np.sum(U * U) + np.sum(V * V) + np.sum(W * W)),
                                                    rel=1e-12)


def test_admission_respects_the_budget(evp):
    from paper_1803_09563_gb300 import serve
    reqs = [serve.Request(arrival_ms=0.0, rid=i, n=32, Wi=1.0, Bi=0.2, beta=0.5, steps=3, seed=i) for i in range(5)]
    L = 2 * np.pi
    one = evp.evp_state_bytes(evp.make_grid(32, 32, 32, L, L, L), evp.EVP_SARAMITO,
                              evp.make_params(Re=100.0, Wi=1.0, beta=0.5, Bi=0.2, precision=evp.EVP_FP32))
    res, rep = serve.Server(budget_bytes=2 * one + one // 2).run(reqs)
    assert rep['requests'] == 5
    assert rep['max_resident'] == 2
    assert rep['p99_ms'] >= rep['p50_ms'] > 0


def test_graph_replay_equals_direct_launches(evp):
    from paper_1803_09563_gb300 import inputs
    n, L = 32, 2 * np.pi
    geo = inputs.geometry(n, n, n, L, L, L)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, 11, 4), 1.0)
    out = []
    for graph in (False, True):
        sim = evp.Simulation(evp.make_grid(n, n, n, L, L, L), 'saramito',
                             evp.make_params(Re=100.0, Wi=2.0, beta=0.5, Bi=0.3, precision=evp.EVP_FP32))
        sim.set_state(U, V, W)
        if graph:
            evp.evp_set_graph(sim.handle, True)
        for _ in range(5):          # both buffer parities, replayed more than once
            sim.step(1e-3)
        sim.sync()
        out.append([sim.get(f) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W, evp.EVP_P, evp.EVP_BXX, evp.EVP_BYZ)])
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_small_requests_do_not_wait_for_large_grids(evp):
    """Each size class steps as soon as its own previous step ends: 32^3 requests
    served beside a long 128^3 one see step latencies below the 128^3 steps (in
    lock-step ticks every step would last at least as long as the largest)."""
    from paper_1803_09563_gb300 import serve
    reqs = [serve.Request(arrival_ms=0.0, rid=0, n=128, Wi=1.0, Bi=0.3, beta=0.5, steps=60, seed=1)]
    reqs += [serve.Request(arrival_ms=0.5 * i, rid=1 + i, n=32, Wi=1.0, Bi=0.3, beta=0.5, steps=20, seed=2 + i)
             for i in range(6)]
    _, rep = serve.Server(budget_bytes=8 << 30, result_fields=()).run(reqs)
    assert rep['requests'] == 7
    small, big = rep['by_size']['32'], rep['by_size']['128']
    assert small['request_steps'] == 6 * 20 and big['request_steps'] == 60
    assert small['p50_ms'] < big['p50_ms'] and small['p99_ms'] < big['p99_ms'], rep['by_size']
    assert rep['queue_p99_ms'] is not None
