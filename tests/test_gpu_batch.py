"""Batched steps (evp_batch_*): members of different grids, models and
parameters advanced with one launch per kernel phase must give, bit for bit, what
each member's own evp_step gives; admission follows the batch's rules and
budget; the autotuner's pick must time within noise of an exhaustive sweep, and
every tile configuration must give the same bits."""

import numpy as np
import pytest

from paper_1803_09563_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ('U', 'V', 'W', 'P', 'BXX', 'BXY', 'BXZ', 'BYY', 'BYZ', 'BZZ')


def member(evp, case, precision, seed):
    """A state of one of the mixed test cases with random solenoidal velocity,
    SPD conformation and pressure."""
    nx, ny, nz, walls, model, extra = case
    ly = 2.0 if walls else 2 * np.pi
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, seed, 3), 1.0)
    if walls:
        U = U + inputs.poiseuille(geo)[0]
    B = inputs.random_conformation(geo, seed + 1, amp=0.3)
    p = np.random.default_rng(seed + 2).standard_normal((nz, ny, nx)) * 0.1
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls), model,
                         evp.make_params(Re=2.0, Wi=0.8, beta=0.4, precision=precision, **extra))
    sim.set_state(U, V, W, p, B)
    return sim


CASES = [
    (32, 32, 32, False, 'saramito', {'Bi': 0.4}),
    (48, 24, 18, False, 'oldroyd_b', {}),
    (36, 20, 16, True, 'fene_p', {'L2': 60.0, 'dpdx': 0.5}),
    (32, 32, 32, False, 'fene_p', {'L2': 60.0, 'abc_amp': 0.7, 'abc_k': 2.0}),
    (64, 12, 24, True, 'saramito', {'Bi': 0.2}),
    (32, 32, 32, False, 'saramito', {'Bi': 0.9}),
]


def snapshot(evp, sim):
    names = [getattr(evp, 'EVP_' + f) for f in FIELDS]
    names += [evp.EVP_RT_XX + c for c in range(6)] + [evp.EVP_NH_X + c for c in range(3)]
    return [sim.get(f) for f in names]


@pytest.mark.parametrize('prec', ['fp32', 'fp64'])
@pytest.mark.parametrize('graph', [False, True])
def test_batch_step_equals_each_member_alone_bitwise(evp, prec, graph):
    precision = evp.EVP_FP32 if prec == 'fp32' else evp.EVP_FP64
    dts = [1e-3, 2e-3, 1.5e-3, 1e-3, 2e-3, 1.2e-3]
    alone = []
    for i, case in enumerate(CASES):
        sim = member(evp, case, precision, 10 + 7 * i)
        if graph:
            evp.evp_set_graph(sim.handle, True)
        for _ in range(3):
            sim.step(dts[i])
        sim.sync()
        alone.append(snapshot(evp, sim))
        sim.close()
    batch = evp.Batch(precision)
    evp.evp_batch_set_graph(batch.handle, graph)
    sims = [member(evp, case, precision, 10 + 7 * i) for i, case in enumerate(CASES)]
    for sim, dt in zip(sims, dts):
        batch.admit(sim, dt)
    assert batch.info()[0] == len(CASES)
    for _ in range(3):           # both buffer parities; the first is replayed again
        batch.step()
    for i, sim in enumerate(sims):
        code, bits, _ = sim.sync(raise_on_error=False)
        assert code == 0
        for a, b in zip(alone[i], snapshot(evp, sim)):
            assert np.array_equal(a, b), (i, CASES[i][:5])
    batch.close()
    for sim in sims:
        sim.close()


def test_membership_changes_and_rules(evp):
    precision = evp.EVP_FP32
    sims = [member(evp, CASES[k], precision, 40 + k) for k in range(3)]
    ref = [member(evp, CASES[k], precision, 40 + k) for k in range(3)]
    batch = evp.Batch(precision, budget_bytes=10 << 30)
    batch.admit(sims[0], 1e-3)
    batch.admit(sims[1], 1e-3)
    batch.step()
    for r in ref[:2]:
        r.step(1e-3)
    # a member cannot step on its own
    with pytest.raises(evp.EvpError) as e:
        sims[0].step(1e-3)
    assert e.value.code == evp.EVP_ERR_STATE
    # the third joins, the first leaves and steps alone again
    batch.admit(sims[2], 1e-3)
    batch.evict(sims[0])
    batch.step()
    for r in ref[1:]:
        r.step(1e-3)
    sims[0].step(1e-3)
    ref[0].step(1e-3)
    for s, r in zip(sims, ref):
        for a, b in zip(snapshot(evp, s), snapshot(evp, r)):
            assert np.array_equal(a, b)
    # rules: another precision, a second batch, the budget
    other = member(evp, CASES[0], evp.EVP_FP64, 50)
    with pytest.raises(evp.EvpError) as e:
        batch.admit(other, 1e-3)
    assert e.value.code == evp.EVP_ERR_ARG
    with pytest.raises(evp.EvpError) as e:
        batch.admit(sims[1], 1e-3)
    assert e.value.code == evp.EVP_ERR_ARG
    n, used = batch.info()
    tight = evp.Batch(precision, budget_bytes=used // 2)
    with pytest.raises(evp.EvpError) as e:
        tight.admit(sims[0], 1e-3)
    assert e.value.code == evp.EVP_ERR_OOM
    newt = evp.Simulation(evp.make_grid(32, 32, 32, 6.0, 6.0, 6.0, False), 'newtonian',
                          evp.make_params(Re=2.0, precision=precision))
    with pytest.raises(evp.EvpError):
        batch.admit(newt, 1e-3)
    # destroying a member state evicts it
    sims[2].close()
    assert batch.info()[0] == 1
    batch.step()
    for x in [tight, batch] + sims + ref + [other, newt]:
        x.close()


def test_tile_configurations_give_the_same_bits(evp):
    """The tile configuration moves work between CTAs, never changes a cell's
    arithmetic."""
    precision = evp.EVP_FP32
    grid_case = CASES[0]
    out = []
    for cfg in ((0, 0, 0, 0, 0), (1, 32, 1, 1, 4), (8, 2, 2, 3, 8), (32, 1, 2, 4, 16)):
        sim = member(evp, grid_case, precision, 61)
        evp.evp_tile_config_set(sim.grid, precision, 'saramito', cfg)
        assert evp.evp_tile_config_get(sim.grid, precision, 'saramito').as_tuple()[:1] != (0,)
        batch = evp.Batch(precision)
        batch.admit(sim, 1e-3)
        batch.step()
        batch.step()
        out.append(snapshot(evp, sim))
        batch.close()
        sim.close()
    evp.evp_tile_config_set(evp.make_grid(32, 32, 32, 2 * np.pi, 2 * np.pi, 2 * np.pi, False), precision,
                            'saramito', (0, 0, 0, 0, 0))
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert np.array_equal(a, b)
    with pytest.raises(evp.EvpError):
        evp.evp_tile_config_set(evp.make_grid(32, 32, 32, 1.0, 1.0, 1.0, False), precision, 'saramito',
                                (64, 0, 0, 0, 0))


def test_autotuner_matches_exhaustive_sweep(evp):
    """On a 32^3 FP32 Saramito box: the coordinate-descent tuner times fewer
    configurations than the exhaustive sweep and its pick, re-timed beside the
    sweep's, is within 10 % (plus 5 us for timing noise) of it."""
    n, L = 32, 2 * np.pi
    grid = evp.make_grid(n, n, n, L, L, L, False)
    prm = evp.make_params(Re=100.0, Wi=1.0, beta=0.5, Bi=0.5, precision=evp.EVP_FP32)
    quick, ms_q, trials_q = evp.evp_tune(grid, 'saramito', prm, exhaustive=False)
    full, ms_f, trials_f = evp.evp_tune(grid, 'saramito', prm, exhaustive=True)
    assert trials_q < trials_f
    tq, tf = [], []
    for _ in range(3):
        tq.append(evp.evp_tile_time(grid, 'saramito', prm, quick, steps=40))
        tf.append(evp.evp_tile_time(grid, 'saramito', prm, full, steps=40))
    assert min(tq) <= 1.10 * min(tf) + 0.005, (quick.as_tuple(), full.as_tuple(), tq, tf)
    # the table keeps the last tuning of this grid
    assert evp.evp_tile_config_get(grid, evp.EVP_FP32, 'saramito').as_tuple() == full.as_tuple()
