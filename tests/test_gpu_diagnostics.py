"""Parity of evp_diagnostics (through the C ABI) with ``oracle.diagnostics`` on the
same seeded fields, for every model, both precisions and both y boundaries.

The integer and extremal results (yielded cells, non-finite cells, min det B,
max tr B) are compared exactly: both sides form them in FP64 from the same
stored values, in the same order of operations.  The sums (kinetic energy) run
in different orders: relative 1e-12.  max |div u| is compared with an absolute
bound of 1e-12 max|u| / min(dx, dy, dz) (it is a difference of face values)."""

import numpy as np
import pytest

import oracle
from oracle import diagnostics as odg
from paper_1803_09563_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(48, 24, 18, False), (36, 20, 16, True), (64, 12, 24, True)]
MODELS = [('newtonian', {}), ('oldroyd_b', {}), ('fene_p', {'L2': 60.0}), ('saramito', None),
          ('neo_hookean', {})]


def _case(evp, shape, model, extra, precision, seed=7, plant=None):
    """A state set from seeded host fields; returns (sim, oracle diagnostics of
    the same fields, grid, host fields (U, V, W, B), oracle Params).  ``plant``
    may edit the host fields before they are set."""
    nx, ny, nz, walls = shape
    ly = 2.0 if walls else 2 * np.pi
    geo = inputs.geometry(nx, ny, nz, 2 * np.pi, ly, 2 * np.pi, walls)
    U, V, W = inputs.scale_max(*inputs.random_solenoidal(geo, seed, 3), 1.0)
    B = inputs.spd_conformation(geo, seed + 1, amp=0.4)
    g = oracle.Grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls)
    re, wi, beta = 2.0, 0.8, 0.4
    if extra is None:
        # Saramito with tau_y at the median |tau^d| of the field: about half the
        # cells yielded
        gm = (1.0 - beta) * (1.0 / re) / wi
        extra = {'Bi': float(np.median(odg.deviatoric_magnitude(B, gm))) * re}
    if walls:
        V = V.copy()
        V[:, -1] = 0.0
    if plant is not None:
        plant(U, V, W, B)
    sim = evp.Simulation(evp.make_grid(nx, ny, nz, geo['lx'], geo['ly'], geo['lz'], walls), model,
                         evp.make_params(Re=re, Wi=wi, beta=beta, precision=precision, **extra))
    sim.set_state(U, V, W, None, None if model == 'newtonian' else B)
    prm = oracle.Params.from_groups(model, Re=re, Wi=wi, beta=beta, **extra)
    rd = (lambda a: a.astype(np.float32).astype(np.float64)) if precision == evp.EVP_FP32 else (lambda a: a)
    ref = odg.diagnostics(rd(U), rd(V), rd(W), None if model == 'newtonian' else [rd(b) for b in B], g, prm)
    return sim, ref, g, (U, V, W, B), prm


def _compare(got, ref, g, umax=1.0):
    assert got['kinetic_energy'] == pytest.approx(ref['kinetic_energy'], rel=1e-12)
    assert abs(got['max_div'] - ref['max_div']) <= 1e-12 * umax / min(g.dx, g.dy, g.dz)
    assert got['min_det_B'] == ref['min_det_B']
    assert got['max_tr_B'] == ref['max_tr_B']
    assert got['max_tr_B_over_L2'] == pytest.approx(ref['max_tr_B_over_L2'], rel=1e-15, abs=0)
    assert got['yielded_cells'] == ref['yielded_cells']
    assert got['yielded_fraction'] == ref['yielded_fraction']
    assert got['nonfinite_cells'] == ref['nonfinite_cells']


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("model,extra", MODELS)
@pytest.mark.parametrize("precision", [0, 1])
def test_diagnostics_match_the_oracle(evp, shape, model, extra, precision):
    sim, ref, g, _, _ = _case(evp, shape, model, extra, precision)
    got = sim.diagnostics()
    _compare(got, ref, g)
    if model == 'saramito':
        assert 0.3 < got['yielded_fraction'] < 0.7
    # a second call on the same fields returns the same bits
    assert sim.diagnostics() == got
    sim.close()


def test_nonfinite_cells_are_counted_and_not_raised(evp):
    def plant(U, V, W, B):
        U[3, 4, 5] = np.nan
        W[15, 19, 35] = np.inf
        B[4][3, 4, 5] = -np.inf             # same cell as the U entry
        B[4][0, 0, 0] = np.nan
    sim, ref, g, _, _ = _case(evp, (36, 20, 16, True), 'oldroyd_b', {}, evp.EVP_FP64, plant=plant)
    got = sim.diagnostics()
    assert ref['nonfinite_cells'] == 3
    assert got['nonfinite_cells'] == 3
    assert got['min_det_B'] == ref['min_det_B'] and got['max_tr_B'] == ref['max_tr_B']
    assert got['yielded_cells'] == ref['yielded_cells']
    # the call reports, it does not raise: the status bits stay clear (evp_sync
    # without its own residual kernel, which would flag the NaN divergence)
    code, bits, _ = sim.sync(raise_on_error=False, max_div=False)
    assert code == evp.EVP_OK and bits == 0
    code, bits, _ = sim.sync(raise_on_error=False)
    assert code == evp.EVP_ERR_NONFINITE and bits == evp.EVP_BIT_NONFINITE
    sim.close()


def test_diagnostics_after_steps_follow_the_oracle(evp):
    """Two RK3 steps of a Saramito channel on both sides, then the diagnostics of
    each side's own state: the continuous quantities agree at the step's
    tolerance and the yielded counts differ by at most the cells whose |tau^d|
    lies within 1e-8 of tau_y (where a rounding difference may flip F > 0)."""
    shape = (32, 16, 16, True)
    sim, _, g, (U, V, W, B), prm = _case(evp, shape, 'saramito', None, evp.EVP_FP64)
    st = oracle.State.rest(g, U, V, W)
    st.B = [b.copy() for b in B]
    dt = 2e-3
    for _ in range(2):
        sim.step(dt)
        st = oracle.rk3_step(st, dt, g, prm)
    sim.sync()
    got = sim.diagnostics()
    ref = odg.diagnostics(st.U, st.V, st.W, st.B, g, prm)
    assert got['kinetic_energy'] == pytest.approx(ref['kinetic_energy'], rel=1e-10)
    assert got['min_det_B'] == pytest.approx(ref['min_det_B'], rel=1e-10)
    assert got['max_tr_B'] == pytest.approx(ref['max_tr_B'], rel=1e-10)
    assert got['max_div'] < 1e-10 and ref['max_div'] < 1e-10
    mag = odg.deviatoric_magnitude(st.B, prm.mu_p / prm.lam)
    band = int(np.count_nonzero(np.abs(mag - prm.tau_y) <= 1e-8 * prm.tau_y))
    assert abs(got['yielded_cells'] - ref['yielded_cells']) <= band
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_member_diagnostics_wait_for_the_batch(evp, precision):
    """A member's diagnostics after a batch step equal those of the same state
    stepped alone (the batch gives the member's own evp_step bit for bit)."""
    shape = (32, 16, 16, True)
    alone = _case(evp, shape, 'saramito', None, precision, seed=11)[0]
    member = _case(evp, shape, 'saramito', None, precision, seed=11)[0]
    batch = evp.Batch(precision)
    batch.admit(member, 1e-3)
    for _ in range(3):
        alone.step(1e-3)
        batch.step()
    a = alone.diagnostics()
    b = member.diagnostics()
    assert a == b
    batch.evict(member)
    batch.close()
    alone.close()
    member.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_two_phase_state_reads_its_current_buffers(evp, precision):
    """An AB2 drop after two steps: the energy and the conformation extremes are
    those of the fields evp_get_field returns (FP32 fields widened, as the
    reductions do)."""
    nx = ny = nz = 32
    L = 2.0
    grid = evp.make_grid(nx, ny, nz, L, L, L, walls_y=True)
    prm = evp.make_params(Re=10.0, Wi=0.5, beta=0.5, Bi=0.3, precision=precision, integrator=evp.EVP_AB2,
                          mu_ratio=1.0, ls_eps_cells=1.5, sigma=0.1, drho_g=1.0, reinit_every=0)
    sim = evp.Simulation(grid, 'saramito', prm)
    geo = inputs.geometry(nx, ny, nz, L, L, L, True)
    sim.set(evp.EVP_PHI, inputs.sphere_distance(geo, (1.0, 0.0, 1.0), 0.4))
    for _ in range(2):
        sim.step(1e-3)
    sim.sync()
    got = sim.diagnostics()
    U, V, W = (sim.get(f).astype(np.float64) for f in (evp.EVP_U, evp.EVP_V, evp.EVP_W))
    B = [sim.get(f).astype(np.float64)
         for f in (evp.EVP_BXX, evp.EVP_BXY, evp.EVP_BXZ, evp.EVP_BYY, evp.EVP_BYZ, evp.EVP_BZZ)]
    dv = (L / nx) ** 3
    ke = 0.5 * dv * (np.sum(U * U) + np.sum(V * V) + np.sum(W * W))
    assert got['kinetic_energy'] == pytest.approx(ke, rel=1e-12)
    assert got['kinetic_energy'] > 0
    assert got['min_det_B'] == odg.det3_sym(B).min()
    assert got['max_tr_B'] == (B[0] + B[3] + B[5]).max()
    assert 0.0 <= got['yielded_fraction'] <= 1.0 and got['nonfinite_cells'] == 0
    sim.close()
