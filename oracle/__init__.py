"""FP64 CPU oracle for the Eulerian non-Newtonian time step of Izbassarov et al.,
"Computational modeling of multiphase viscoelastic and elastoviscoplastic flows"
(arXiv 1803.09563).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
restatement of the paper's discrete method that the CUDA path is checked against.
It is imported only by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path
(``paper_1803_09563_gb300``) never imports, links or executes anything here, and
nothing here imports the product path.

Everything is numpy float64, vectorised over whole arrays with no blocking or
fusion.  Library primitives used as steps: ``numpy.fft`` (the FFTs of the fast
Poisson solver).  Each function cites the section / equation / table of the paper
it restates.  Where the paper is silent the reading taken is stated in the
docstring ("Reading n"); the CUDA path takes the same numbered readings.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
  grid shifts, centre velocity, velocity gradient ... pinned (brute force, closed forms)
  WENO5 (Sec. 3.1) ................................. pinned (textbook 5th-order formula,
                                                     polynomial exactness, ENO switch,
                                                     convergence order)
  closures (Table 1), stress RHS (Eq. SRM2) ........ pinned (start-up / oscillatory
                                                     shear closed forms, Saramito yield
                                                     time, steady yielded shear, axis
                                                     swaps and mirrors of the cube)
  stress from B (Table 1 inverted) ................. pinned (Oldroyd-B start-up shear,
                                                     FENE-P steady shear: tau_yy = 0,
                                                     tau_xy = mu_p gdot a/F, N1; planted
                                                     slips fail)
  Saramito channel (Sec. 4.1.1, Table 1) ........... pinned (plug half-width y0 of the
                                                     closed form, steady-shear relations
                                                     of the yielded cells, force balance,
                                                     velocity profile of a 1-D root find;
                                                     planted slips fail)
  local artificial diffusion (Sec. 3.1) ............ pinned (sine-mode eigenvalues of the
                                                     stencil, trigger thresholds, wall
                                                     row, conservation)
  momentum RHS (Eq. NS-num1) ....................... pinned (Taylor-Green decay order,
                                                     steady Oldroyd-B Poiseuille, kinetic
                                                     energy conserved by the advection
                                                     form, summation by parts of div tau
                                                     with the velocity gradient and of
                                                     grad p with the divergence, symmetric
                                                     negative viscous forms, 1-D
                                                     variable-viscosity fluxes)
  Poisson solve + projection (Eqs. NS-num2/3) ...... pinned (sine modes, sparse direct
                                                     solve, divergence <= 1e-12)
  RK3 constants (Eq. RK) ........................... pinned (3rd-order convergence on
                                                     a linear ODE closed form; a whole
                                                     step multiplies a shear mode and a
                                                     relaxing uniform conformation by
                                                     the RK3 stability polynomial)
  level set (Eqs. ls-adv, normal, curv, reinit) .... pinned (translation, sphere
                                                     curvature, Heaviside volume, Laplace
                                                     pressure jump of the CSF force,
                                                     mean-free buoyancy)
  AB2 (Eqs. ab2tau, ab2) ........................... pinned (2nd-order convergence; a
                                                     shear mode follows the AB2
                                                     recurrence exactly)
  density-contrast split projection ................ pinned (div-free, uniform-density limit,
                                                     fixed point = sparse variable solve)
  mass-preserving level-set shift .................. pinned (exact undo of a shift,
                                                     volume conservation)
  implicit viscous option (Helmholtz) .............. pinned (operator residual, closed-form
                                                     shear-mode decay, dt^3 local error)
  volume penalisation .............................. pinned (alpha = 0 bitwise, alpha = 1,
                                                     solid block)
  rigid-particle IBM, free motion .................. pinned (Roma moments, linear exactness,
                                                     conservation, convergence, integrals,
                                                     first substep under gravity)
  soft particles ................................... pinned (all-solid and all-fluid limits,
                                                     transport order)
  monitoring quantities ............................ pinned (Fourier-mode energy, steady-shear
                                                     det B, library determinant, deviator
                                                     closed forms, yielded cells beyond
                                                     the channel's plug edge y0)

The substep predictors (``rk3_substep(..., predictor_only=True)``,
``ab2.ab2_predictor``) return u* and the updated conformation before the global
projection; the full-size GPU tests evaluate them on windows of the full fields
(``tests/oracle_windows.py``; the window interior equals the full-field result bit
for bit, ``tests/test_oracle_windows.py``).
"""

from .grid import Grid, at  # noqa: F401
from .weno import hj_weno5, weno5_derivative  # noqa: F401
from .models import Params, closure, tau_from_B, rt_local  # noqa: F401
from .stress import centre_velocity, velocity_gradient, stress_rhs, determinant, diffusion_cells  # noqa: F401
from .momentum import advection, laplacian, div_tau, grad_p, momentum_rhs_n  # noqa: F401
from .poisson import divergence, eigenvalues, solve_poisson, project  # noqa: F401
from .step import State, rk3_step, rk3_substep, RK3_ALPHA, RK3_ZETA, RK3_XI  # noqa: F401
from . import levelset  # noqa: F401,E402
from .ab2 import TwoPhase, ab2_step  # noqa: F401,E402
from . import ibm  # noqa: F401,E402
