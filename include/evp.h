/*
 * evp.h -- C ABI of libevp, a GB300 (sm_103a) implementation of the Eulerian
 * non-Newtonian time step of Izbassarov et al., "Computational modeling of
 * multiphase viscoelastic and elastoviscoplastic flows" (arXiv 1803.09563).
 *
 * One call advances a simulation on a staggered uniform Cartesian grid (Sec. 3):
 * the conformation tensor B of Eq. SRM2 with the closures of Table 1 (Oldroyd-B,
 * FENE-P, Saramito EVP), fifth-order WENO advection of B (Sec. 3.1), the
 * momentum predictor with div(tau) (Eq. NS-num1), and the fast Poisson
 * projection (Eqs. NS-num2, NS-num3) with FFTs in the periodic directions and a
 * tridiagonal (Thomas) solve along a wall-normal y, all integrated with the
 * low-storage RK3 scheme of Eq. RK.
 *
 * Conventions shared by every entry point
 *   - Plain C types only.  Device pointers are CUDA device addresses on the
 *     current device; host pointers are ordinary (preferably pinned) memory.
 *   - Field layout: [nz][ny][nx], x fastest, nx*ny*nz elements.  A face
 *     velocity at index i is the one on the +1/2 face of cell i (u at
 *     x = (i+1)dx, v at y = y0 + (j+1)dy, w at z = (k+1)dz); with walls the
 *     face below cell j = 0 is the bottom wall and v[.., ny-1, ..] the top wall.
 *     Centred fields (p, B, phi) sit at cell centres.
 *   - Element type of every field buffer is the state's precision: double for
 *     EVP_FP64, float for EVP_FP32.
 *   - Every function returns an evp_status (EVP_OK = 0).  No exception crosses
 *     the ABI.  On failure evp_last_error() holds a message for the calling
 *     thread.  Kernel-side conditions (non-finite values, FENE-P trace limit,
 *     loss of positive definiteness) raise status bits that evp_sync() returns.
 *   - Asynchrony: evp_step / evp_substep / evp_project / evp_poisson_solve /
 *     evp_stress_rhs enqueue work on the state's stream and return.
 *     evp_set_field / evp_get_field and evp_sync synchronise that stream.
 *   - Threading: a state is used by one host thread at a time.
 */
#ifndef EVP_H
#define EVP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EVP_OK = 0,
    EVP_ERR_ARG = 1,         /* invalid argument (sizes, ids, null pointers)       */
    EVP_ERR_OOM = 2,         /* device allocation failed or arena too small         */
    EVP_ERR_CUDA = 3,        /* a CUDA runtime call failed                          */
    EVP_ERR_NONFINITE = 4,   /* a kernel produced NaN/Inf (raised at evp_sync)      */
    EVP_ERR_UNPHYSICAL = 5,  /* FENE-P tr B >= L^2, or det B < 0 without art_diff (raised at sync) */
    EVP_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                       */
    EVP_ERR_STATE = 7,       /* call not valid in the state's configuration         */
    EVP_ERR_BOUNDS = 8       /* debug build (EVP_DEBUG) only: a kernel's index, range
                                or alignment check failed (raised at evp_sync)       */
} evp_status;

/* status bits accumulated by the kernels, returned by evp_sync */
#define EVP_BIT_NONFINITE   0x1u
#define EVP_BIT_TRACE_LIMIT 0x2u   /* FENE-P: tr B >= L^2 (Table 1 closure singular)  */
#define EVP_BIT_DET_NEG     0x4u   /* det B < 0: B lost positive definiteness (Sec 3.1) */
#define EVP_BIT_BOUNDS      0x8u   /* debug build only: a checked access of a stencil
                                      kernel was out of its field, out of the kernel's
                                      shared memory or misaligned; it was skipped      */

/* Grid (Sec. 3): uniform spacing lx/nx, ly/ny, lz/nz.  x and z are periodic;
 * y is periodic (walls_y = 0) or bounded by no-slip walls at y = -ly/2 and
 * +ly/2 (walls_y = 1).  nx and nz (and ny when periodic) must be of the form
 * 2^a 3^b, 8 <= n <= 512; nx even.  With walls 4 <= ny <= 512.             */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    int walls_y;
} evp_grid;

typedef enum {
    EVP_NEWTONIAN = 0,   /* no extra stress (tau = 0)                          */
    EVP_OLDROYD_B = 1,   /* Table 1: B = tau lambda/mu_p + I, F = 1, a = 1    */
    EVP_FENE_P = 2,      /* Table 1: F = L^2/(L^2 - tr B), a = L^2/(L^2 - 3)  */
    EVP_SARAMITO = 3,    /* Table 1: F = a = max(0, 1 - tau_y/|tau^d|)        */
    EVP_NEO_HOOKEAN = 4  /* Table 1: B = tau/G, F = a = 0; G = mu_p/lambda    */
} evp_model;

enum { EVP_FP64 = 0, EVP_FP32 = 1 };
enum { EVP_RK3 = 0, EVP_AB2 = 1 };

/* Dimensionless groups and options.  Scalings (rho = 1): mu_s = beta/Re,
 * mu_p = (1-beta)/Re, lambda = Wi; tau_y = Bi/Re (bi_def = 0, Bi against the
 * viscous stress, Sec. 4.1.3) or tau_y = Bi (bi_def = 1, Bi against rho g L,
 * Sec. 4.2.3).  Body forces (RK3 only): a uniform force dpdx along x (the
 * channel's pressure gradient) and the ABC force
 * abc_amp*(sin kz + cos ky, sin kx + cos kz, sin ky + cos kx), k = abc_k.
 *
 * integrator = EVP_AB2 selects the two-phase drop step of Secs. 3.2.1-3.2.2:
 * a level set phi (phi > 0 outer fluid with the model above, phi < 0 a
 * Newtonian drop of total viscosity mu_ratio/Re), advected by TVD-RK3 + WENO5
 * and re-distanced every reinit_every steps with reinit_iters pseudo-steps
 * (Eq. reinit); mixture viscosities from H(phi) smoothed over ls_eps_cells
 * cells; CSF surface tension sigma (Eq. fLS) and Boussinesq buoyancy drho_g
 * (minus its domain mean) along +y; AB2 for B and u (Eqs. ab2tau, ab2) with a
 * forward-Euler first step; pressure from one projection per step.            */
typedef struct {
    double Re, Wi, beta, Bi, L2;
    int bi_def;
    double dpdx;
    double abc_amp, abc_k;
    int precision;      /* EVP_FP64 or EVP_FP32 (wall-normal Thomas sweeps: FP64 for EVP_FP64,
                           double-single, two floats of about 48 bits, for EVP_FP32) */
    int integrator;     /* EVP_RK3 (Eq. RK) or EVP_AB2 (two-phase step)                 */
    double mu_ratio;    /* AB2: drop total viscosity / outer total viscosity            */
    double ls_eps_cells;/* AB2: half-width of the smoothed Heaviside, in cells          */
    double sigma;       /* AB2: surface tension                                          */
    double drho_g;      /* AB2: buoyancy, density difference times gravity               */
    int reinit_every;   /* AB2: re-distance every this many steps (0: never)            */
    int reinit_iters;   /* AB2: pseudo-time steps per re-distancing (dtau = dx/2)       */
    double rho_ratio;   /* AB2: 0 = Boussinesq drop (drho_g); > 0 = drop / outer density
                           ratio, solved with the constant-coefficient splitting of
                           Eqs. poisson-LS and projection-LS, rho_0 = the smaller density */
    double gravity;     /* gravity g along -y: AB2 with rho_ratio > 0, and free IBM particles */
    int penalization;   /* RK3: volume-penalisation IBM for fixed obstacles (Sec. 3.3.2):
                           u** = (1 - alpha) u* before each projection (Eq. forceAdded),
                           alpha = solid fraction of the control volume around each
                           velocity node, set with EVP_SOLID_X/Y/Z (zero at init)       */
    double art_diff;    /* local artificial diffusion of B (Sec. 3.1), 0 = off: where
                           det B < 0, or tr B >= 0.95 L^2 for FENE-P (tested on the B the
                           stress right-hand side is formed from), art_diff times the
                           7-point Laplacian of B is added to that right-hand side.  The
                           paper gives no value ("tuned" per case).  Explicit: keep
                           art_diff*dt*(2/dx^2 + 2/dy^2 + 2/dz^2) below about 1          */
    int ls_mass_iters;  /* AB2: 0 = off; else after each level-set step phi is shifted
                           uniformly, phi + d, with d from this many Newton iterations on
                           the smoothed drop volume sum (1 - H(phi)) dV, so that it keeps
                           its value of the first step (a mass-preserving reading of the
                           interface-correction level set the paper cites)              */
    int viscous_implicit;/* RK3: 0 = explicit viscous term (advective weights); 1 = Eq.
                           NS-num1 read literally: alpha^k mu_s lap u at levels k-1
                           (explicit) and k (implicit), i.e. one Helmholtz solve
                           u* - alpha^k dt mu_s lap u* = rhs per velocity component and
                           substep (FFT in x, z; Thomas along a wall-bounded y).
                           Not with penalization.                                       */
    int soft_particles; /* RK3, model EVP_NEO_HOOKEAN: soft particles in one continuum
                           (Sec. 3.3.2): the solid volume fraction phi_s (field EVP_PHI,
                           0 fluid .. 1 solid) is advected like B (WENO5, RK3 weights)
                           and the extra stress is phi_s G (B - I), G = mu_p/lambda; the
                           surrounding fluid is Newtonian (mu_s)                        */
    int thomas_fp64;    /* EVP_FP32 states with walls: 0 (default) = the wall-normal Thomas
                           sweeps in double-single arithmetic (pairs of floats, about 48
                           significant bits, on the FP32 pipes); 1 = in FP64.  Both give
                           the FP32 result of the FP64 solve to within an ulp; FP64
                           states always sweep in FP64                                 */
    double reserved[4];
} evp_params;

/* Field identifiers for evp_set_field / evp_get_field */
typedef enum {
    EVP_U = 0, EVP_V = 1, EVP_W = 2, EVP_P = 3,
    EVP_BXX = 4, EVP_BXY = 5, EVP_BXZ = 6, EVP_BYY = 7, EVP_BYZ = 8, EVP_BZZ = 9,
    EVP_RT_XX = 10, /* ... EVP_RT_XX+5: RK3 history RT^{k-2} (Eq. RK-rt)          */
    EVP_NH_X = 16,  /* ... EVP_NH_X+2: RK3 history of -div(uu)+viscous+force     */
    EVP_PSI = 19,   /* last projection variable psi (read only)                  */
    EVP_PHI = 20,   /* AB2: level set phi at cell centres; RK3 with soft_particles:
                       the solid volume fraction phi_s                              */
    EVP_SOLID_X = 21, EVP_SOLID_Y = 22, EVP_SOLID_Z = 23,
                    /* penalization states: solid fractions alpha at u, v, w nodes */
    EVP_NFIELDS = 24
} evp_field;

typedef struct evp_state_s evp_state;

/* Bytes of device memory a state with this configuration needs (its arena). */
size_t evp_state_bytes(const evp_grid* grid, evp_model model, const evp_params* params);

/* Create a state: B = I (tau = 0), u = p = 0, histories zero.
 *   stream: a cudaStream_t, or NULL to let the state create its own stream.
 *   arena:  NULL to let the library allocate evp_state_bytes() on the device,
 *           or a caller-owned device buffer of at least arena_bytes >=
 *           evp_state_bytes(), 256-byte aligned (as cudaMalloc returns); the
 *           caller keeps ownership and must keep it alive until evp_destroy.
 *           The state never retains any other caller pointer.
 * Errors: EVP_ERR_ARG (bad sizes/model/params), EVP_ERR_OOM, EVP_ERR_CUDA.    */
int evp_init(const evp_grid* grid, evp_model model, const evp_params* params,
             void* stream, void* arena, size_t arena_bytes, evp_state** out);

/* Release the state (and its arena and stream if the library created them). */
int evp_destroy(evp_state* s);

/* Copy a whole field (nx*ny*nz elements of the state's precision) into / out of
 * the state.  src/dst are device pointers when *_on_device != 0, host pointers
 * otherwise.  Synchronous with respect to the host.  EVP_PSI is read only.    */
int evp_set_field(evp_state* s, int field, const void* src, int src_on_device);
int evp_get_field(evp_state* s, int field, void* dst, int dst_on_device);

/* Several fields at once: n copies as evp_set_field / evp_get_field would make
 * (fields[i] <-> bufs[i], each nx*ny*nz elements of the state's precision), all
 * enqueued on the state's stream, then one synchronisation.  Host buffers that
 * are page-locked (cudaHostAlloc / pinned) copy asynchronously at full link
 * speed.  The arrays fields and bufs (n entries) are read during the call only.
 * Errors: EVP_ERR_ARG (n < 0, null arrays or buffers, unknown field, EVP_PSI in
 * evp_set_fields), in which case nothing is copied.                          */
int evp_set_fields(evp_state* s, int n, const int* fields, const void* const* srcs, int src_on_device);
int evp_get_fields(evp_state* s, int n, const int* fields, void* const* dsts, int dst_on_device);

/* One step with its inputs and outputs on the host, nothing waited for: the n_in
 * copies into the state (as evp_set_fields), one evp_step of size dt, then the
 * n_out copies out of the state (as evp_get_fields), all enqueued in this order
 * on the state's stream and left running.  Host buffers should be page-locked
 * (then the copies are asynchronous; pageable buffers make the call wait for
 * them); the caller keeps them untouched until the stream is synchronised
 * (evp_sync).  Several states on different streams overlap one state's copies
 * with another's step (the paper has no counterpart).
 * Errors: as evp_set_fields / evp_step / evp_get_fields, found before anything
 * is enqueued when they concern the arguments.                               */
int evp_step_io(evp_state* s, double dt, int n_in, const int* in_fields, const void* const* in_srcs, int n_out,
                const int* out_fields, void* const* out_dsts);

/* One full RK3 time step of size dt (Sec. 3.3.1, Eqs. RK-rt..NS-num3, RK):
 * three substeps, each B update (Eq. rk3tau), momentum predictor (Eq. rk3),
 * Poisson solve (Eq. NS-num2) and correction (Eq. NS-num3).  Asynchronous.   */
int evp_step(evp_state* s, double dt);

/* Replay evp_step from CUDA graphs (RK3 states): the first step for a given dt
 * and buffer parity is captured on the state's stream and instantiated, later
 * steps launch the graph, cutting the per-step host cost of the 24 kernel
 * launches (small grids, many concurrent simulations).  Not while kernel timing
 * is on.  If the stream cannot be captured the state falls back to direct
 * launches.  EVP_ERR_STATE for AB2 states.  Off by default.                    */
int evp_set_graph(evp_state* s, int enable);

/* Programmatic dependent launch of the step's kernels when they are launched
 * directly (on by default; a graph-replayed step uses plain launches, which
 * measured faster there): each kernel may be scheduled while the previous one is
 * finishing and waits inside (griddepcontrol.wait) until that kernel's results
 * are visible, which hides launch latency between the 24 kernels of an RK3 step.
 * Results are identical either way.  Synchronises the state's stream; captured
 * step graphs are rebuilt on the next step.  The paper has no counterpart.      */
int evp_set_pdl(evp_state* s, int enable);

/* NVTX ranges for profilers (Nsight Systems timelines, Nsight Compute's --nvtx
 * filters); off by default.  When on, evp_step and evp_substep each open a range
 * ("evp_step", "evp_substep k"; "evp_step graph replay" around a replayed
 * step graph, whose kernels carry no range of their own) and every directly
 * launched kernel of the step opens one named as in evp_kernel_name.  Host-side
 * markers only: results are identical either way, and without a profiler
 * attached a range costs a function-pointer test.  The paper has no counterpart. */
int evp_set_nvtx(evp_state* s, int enable);

/* Rigid spherical particles coupled to the RK3 step by the discrete-forcing
 * immersed boundary method of Sec. 3.3.2 (Eqs. IBM a-d with the multi-direct
 * forcing of Eq. CoVe2, iters iterations per substep, 3 in the paper): after u*
 * is formed, the velocity interpolated with the three-point Roma kernel to
 * Lagrangian points on each sphere (retracted by 0.3 dx, spiral lattice, about
 * one point per dx^2 of surface) is driven towards the surface velocity
 * U_p + omega_p x r, and u** replaces u* in the projection.
 *   desc: host, n x 11 doubles per particle: centre x, y, z; radius; U_p (3);
 *         omega_p (3); density ratio rho_p/rho_f.  A ratio of 0 prescribes the
 *         motion (U_p, omega_p constant, the centre moves with U_p); a positive
 *         ratio makes the sphere free: the Newton-Euler equations of the paper
 *         (Eqs. NewtonEulerWim1/2, with the inner-fluid integrals, gravity
 *         evp_params.gravity along -y, no collisions) advance U_p, omega_p and the
 *         centre every substep.  n = 0 removes the particles.
 * Needs cubic cells, radius >= 2 dx, 2 (R + 2 dx) below the periodic lengths and
 * (walls) |y_c| + R + 2 dy <= ly/2.  Synchronises; the step graph is rebuilt.
 * Errors: EVP_ERR_ARG, EVP_ERR_STATE (AB2 states), EVP_ERR_OOM.               */
int evp_set_particles(evp_state* s, int n, const double* desc, int iters);

/* Per particle, 15 doubles into out (host): current centre (3), velocity (3),
 * angular velocity (3), then the force (3) and torque about the centre (3) that
 * the IBM exerted on it in the last substep, -sum F_l dV_l and
 * -sum r_l x F_l dV_l.  n must equal the count set.  Synchronises.             */
int evp_get_particles(evp_state* s, int n, double* out);

/* With integrator EVP_AB2, evp_step is one two-phase AB2 step of size dt
 * (level set, re-distancing when due, interface force, B and u updates,
 * projection with dt); steps are counted from evp_init.                       */

/* Substep k = 0, 1, 2 of the RK3 scheme alone (Eq. RK constants alpha^k,
 * zeta^k, xi^k; EVP_ERR_STATE for an AB2 state).  For k > 0 the histories RT^{k-2} and N^{k-2} are the ones in
 * the state (set them with evp_set_field to reproduce an arbitrary substep).  */
int evp_substep(evp_state* s, double dt, int k);

/* Project the current velocity onto the discretely divergence-free space:
 * lap(phi) = div u, u <- u - grad(phi) (Eqs. var-poisson, projection with
 * dt = 1).  The pressure field is left unchanged.  Asynchronous.              */
int evp_project(evp_state* s);

/* Solve lap(psi) = rhs with the state's fast Poisson solver (FFT in periodic
 * directions, Thomas along a wall-bounded y; Eq. NS-num2).  rhs and psi
 * are device buffers of nx*ny*nz elements (state precision); rhs may equal psi.
 * Periodic: the mean of rhs is ignored and psi has zero mean.  Walls: the
 * (kx, kz) = (0, 0) system is pinned by psi = 0 in its first row.             */
int evp_poisson_solve(evp_state* s, const void* rhs, void* psi);

/* No-allocation variant of evp_poisson_solve (the paper has no counterpart).
 * For callers that cannot allocate device memory where they need a solve: code
 * that runs while a stream is being captured into a CUDA graph, plugins whose
 * host framework owns all device memory, or processes held to a fixed memory
 * budget.  It needs no evp_state and calls no cudaMalloc/cudaFree or any other
 * allocating routine.  All scratch (spectral buffer, FFT tables, Thomas pivots
 * and the FP64 sweep buffer) lives in one file-scope device array of 8 MiB that
 * every GPU loading the library holds until the process exits.
 *   grid:      as for evp_init; the solve's scratch must fit in the 8 MiB array
 *              (for example 64^3 in FP64 or 96^3 in FP32, periodic), else
 *              EVP_ERR_ARG with a message giving the bytes needed.
 *   precision: EVP_FP64 or EVP_FP32 (element type of rhs and psi).
 *   rhs, psi:  device buffers of nx*ny*nz elements, caller-owned; rhs may equal psi.
 *   stream:    cudaStream_t to run on (NULL = legacy default stream).
 * The result is that of evp_poisson_solve on the same grid.  Calls that are not
 * being captured look up the array's device address (cudaGetSymbolAddress) with
 * the current device; the first call on a device may load the module there.  A
 * call whose grid or precision differs from the previous call's on that device
 * (or that finds the array moved, after cudaDeviceReset) uploads its tables into
 * the array.  Make the first call and such calls before any stream capture: a
 * captured call that would need the lookup or an upload returns EVP_ERR_STATE.  All calls on a
 * device share the array and it keeps the last call's contents (nothing in it
 * needs to start at zero): calls that overlap on the GPU, on any streams, race
 * and give wrong results.  A CUDA graph that holds this call reads the tables in
 * place, so it stays valid only until the next call on that device with another
 * grid or precision, even when the calls never overlap.
 * Asynchronous on ``stream``.                                                    */
int evp_poisson_solve_static(const evp_grid* grid, int precision, const void* rhs, void* psi, void* stream);

/* Evaluate RT = (aI - F B)/lambda - (u.grad B - B.grad u - grad u^T.B) of Eq. rt
 * at the current state into rt (device, 6*nx*ny*nz elements, component-major
 * in the order xx, xy, xz, yy, yz, zz).                                        */
int evp_stress_rhs(evp_state* s, void* rt);

/* Wait for the state's stream.  Returns EVP_ERR_NONFINITE / EVP_ERR_UNPHYSICAL
 * when kernels raised the matching bits since the last sync (bits in *bits),
 * else EVP_OK.  With art_diff > 0, EVP_BIT_DET_NEG is reported in *bits but is
 * not an error: det B < 0 is then the condition the diffusion treats.
 * max_div (may be NULL): when given, a kernel evaluates max |div u| of the
 * state's current velocity (after a step or evp_project, the last projection's
 * output) in FP64 on the stored values, which *max_div receives; a non-finite
 * divergence sets EVP_BIT_NONFINITE.  The steps themselves compute no residual.
 * Bits are cleared afterwards.                                                 */
int evp_sync(evp_state* s, unsigned* bits, double* max_div);

/* Monitoring quantities of the current state (the paper monitors flow
 * histories such as the centre-line velocity, B_xx and the yielded region,
 * Sec. 4, and names loss of positive definiteness of B as the failure mode,
 * Sec. 3.1; these reductions are the library's summary of that state).  All
 * are evaluated in FP64 on the stored values (FP32 states are widened first);
 * every sum runs in a fixed order, so repeated calls on the same fields give
 * the same bits.                                                               */
typedef struct evp_diag {
    double kinetic_energy;   /* 1/2 dx dy dz sum over all stored faces of u^2 + v^2 + w^2
                                (rho = 1; with walls the wall v faces hold 0)          */
    double max_div;          /* max |div u| over the cells whose divergence is finite
                                (as evp_sync's max_div)                               */
    double min_det_B;        /* min over the cells of det B; +inf for EVP_NEWTONIAN  */
    double max_tr_B;         /* max over the cells of tr B; 0 for EVP_NEWTONIAN      */
    double max_tr_B_over_L2; /* FENE-P: max tr B / L^2 (the closure is singular at 1);
                                0 for the other models                                 */
    double yielded_fraction; /* EVP_SARAMITO: fraction of the cells with F > 0 of
                                Table 1, i.e. |tau^d| > tau_y with tau = mu_p/lambda
                                (B - I); two-phase states form mu_p from the Heaviside
                                of the last step's level set (0 before the first
                                step).  1 for Oldroyd-B and FENE-P, 0 for Newtonian
                                and neo-Hookean (no yield surface)                     */
    unsigned long long nonfinite_cells; /* cells where u, v or w of the cell's faces
                                (i, j, k) or a component of B is NaN or infinite    */
    unsigned long long yielded_cells;   /* the count behind yielded_fraction         */
} evp_diag;

/* Fill *out with the current state's monitoring quantities.  Waits for the
 * state's stream (and its batch's, for a batch member) and then for the
 * reduction; allocates nothing (the state's arena holds the block partials).
 * Non-finite cells are reported, not raised: the status bits of evp_sync are
 * left as they are.
 * Errors: EVP_ERR_ARG (null pointers), EVP_ERR_CUDA.                           */
int evp_diagnostics(evp_state* s, evp_diag* out);

/* Self-test of the current device (the paper has no counterpart): checks the
 * integer-operation conversions between binary32 and binary64 that the FP64
 * divergence residual and the FP32 Thomas sweep use against the hardware
 * conversion instructions, over all 2^32 binary32 patterns (widening) and 2^30
 * binary64 patterns around the binary32 range, including every kind of rounding
 * tie (narrowing).  Results must agree bit for bit, except that values in the
 * binary32 subnormal range give a signed zero and a NaN gives some NaN.
 * *mismatches receives the number of failures (0 expected).  Synchronous;
 * allocates 16 bytes.                                                          */
int evp_selftest(unsigned long long* mismatches);

/* ---------------------------------------------------------------- batches
 * Many simulations advanced together (the paper has no counterpart: it runs one
 * simulation per job).  A batch advances every member state by one RK3 step of
 * that member's dt per evp_batch_step, with one launch per kernel phase for all
 * members: the stress update and the momentum predictor as persistent kernels
 * over a device work list of (member, tile) that may mix grid sizes, the
 * Poisson passes and the correction once per group of members on the same grid
 * (the FFT kernels are specialised by length).  Every member computes exactly
 * what evp_step computes for it alone (bit for bit).  Steps replay a CUDA graph
 * per membership, dt and buffer parity (captured on first use).
 * Members: RK3 states with a stress (Oldroyd-B, FENE-P, Saramito) of the
 * batch's precision, without penalisation, particles, soft particles, the
 * implicit viscous option or artificial diffusion; at most 64 members.  While a
 * state is a member its evp_step / evp_substep return EVP_ERR_STATE; field
 * copies and evp_sync on it first wait for the batch's stream.               */
typedef struct evp_batch_s evp_batch;

/* Tile configuration of the batched kernels for one grid: z planes per work item
 * of the stress and momentum kernels, resident CTAs per SM of their persistent
 * grids (at most 2 and 4 in FP32, 1 and 2 in FP64), and kx columns per block of
 * the column FFT passes (4, 8 or 16; 16 only in FP32).  0 in a field: the
 * default (the heuristic of the single-state launches).                       */
typedef struct {
    int stress_kz, momentum_kz;
    int stress_ctas_per_sm, momentum_ctas_per_sm;
    int fft_cols;
} evp_tile_config;

/* Create an empty batch.  precision: EVP_FP64 or EVP_FP32, of every member.
 * budget_bytes: admission limit on the sum of the members' evp_state_bytes (0:
 * none).  stream: a cudaStream_t the batch runs on, or NULL to create one.   */
int evp_batch_create(int precision, size_t budget_bytes, void* stream, evp_batch** out);
/* Add a state with its time step dt.  Waits for the state's stream.  Errors:
 * EVP_ERR_ARG (state not eligible, see above, or already a member of a batch),
 * EVP_ERR_OOM (budget or member count exceeded; nothing changes).             */
int evp_batch_admit(evp_batch* b, evp_state* s, double dt);
/* Remove a member (waits for the batch's stream); the state stays valid and
 * can step on its own again.  EVP_ERR_ARG if it is not a member.              */
int evp_batch_evict(evp_batch* b, evp_state* s);
/* One RK3 step of every member, asynchronous on the batch's stream.           */
int evp_batch_step(evp_batch* b);
/* Members and bytes admitted (either pointer may be NULL).                    */
int evp_batch_info(const evp_batch* b, int* members, size_t* bytes);
/* Replay steps from CUDA graphs (1, the default) or launch them directly (0). */
int evp_batch_set_graph(evp_batch* b, int enable);
/* Evict every member, release the batch (and its stream if it created it).    */
int evp_batch_destroy(evp_batch* b);

/* Self-written tile autotuner: times batched steps of a scratch state of this
 * grid, model and parameters (one member, B = I and a smooth solenoidal
 * velocity) under candidate tile configurations and keeps the fastest in a
 * process-wide table keyed by (grid, precision, model), which batches use for
 * members on that grid from their next membership change on.
 *   exhaustive = 0: coordinate descent over the five fields, each swept with the
 *   others held, twice round; 1: every combination.  best receives the chosen
 *   configuration, best_ms its time per step, trials the configurations timed.
 * Synchronous; allocates a scratch state.                                     */
int evp_tune(const evp_grid* grid, evp_model model, const evp_params* params, int exhaustive,
             evp_tile_config* best, double* best_ms, int* trials);
/* Time per step (ms, median of 3 runs of `steps` graph-replayed steps) of the
 * scratch one-member batch of evp_tune under one configuration.  Synchronous.  */
int evp_tile_time(const evp_grid* grid, evp_model model, const evp_params* params, const evp_tile_config* cfg,
                  int steps, double* ms_per_step);
/* The configuration batches use for this grid: the tuned (or set) one, else the
 * default with every field filled in.                                         */
int evp_tile_config_get(const evp_grid* grid, int precision, evp_model model, evp_tile_config* out);
/* Put a configuration in the table (zero fields: defaults); all fields zero
 * removes the grid's entry.  Batches pick it up at their next membership
 * change.  EVP_ERR_ARG when a field is out of range.                          */
int evp_tile_config_set(const evp_grid* grid, int precision, evp_model model, const evp_tile_config* cfg);

/* Measured peak of the plain (non-tensor) FMA pipe of the current device, the
 * roofline of arithmetic-bound kernels (the paper has no counterpart): every
 * thread of 8 blocks per SM runs eight independent chains of fused multiply-adds
 * (EVP_FP32: the packed two-lane f32x2 instruction the stress kernel uses;
 * EVP_FP64: the double-precision FMA), timed with CUDA events on the legacy
 * stream; *flops_per_s receives the best of three timed launches after a
 * warm-up, counting an FMA as two operations.  Synchronous; about 0.2 s;
 * allocates 16 bytes.  The rate follows the SM clock at the time.              */
int evp_fma_peak(int precision, double* flops_per_s);

/* Per-kernel timing with CUDA events on the state's stream (off by default).
 * evp_kernel_times fills up to n entries of accumulated milliseconds and
 * launch counts (synchronises); evp_kernel_name names entry i.              */
int evp_kernel_timing(evp_state* s, int enable);
int evp_kernel_times(evp_state* s, double* ms, long long* launches, int n);
const char* evp_kernel_name(int i);
int evp_num_kernels(void);

/* Message of the last failing call on this thread ("" if none). */
const char* evp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EVP_H */
