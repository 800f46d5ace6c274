// Internal declarations shared by the libevp translation units: grid index maps,
// kernel argument blocks and the launch functions of each kernel family.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "evp.h"

#include <vector>

namespace evp {

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// Kernel identifiers for the per-kernel event timing.
enum KernelId {
    K_STRESS = 0,     // S1 + S2: centre velocity/gradient, WENO5 advection, closure, B update
    K_MOMENTUM,       // S3: momentum predictor u*
    K_DIV_FFTX,       // S4 + S5(x): Poisson right-hand side fused into the x real-to-complex FFT
    K_FFT_Z_FWD,      // S5(z): forward complex FFT along z
    K_SOLVE_Y,        // S5(y) + S6 + S7(y), periodic y: FFT, modal division, inverse FFT
    K_THOMAS,         // S6, walls: FP64 tridiagonal solve per (kx, kz)
    K_FFT_Z_INV,      // S7(z): inverse complex FFT along z
    K_IFFTX,          // S7(x): complex-to-real inverse FFT along x -> psi
    K_CORRECT,        // S8: u = u* - c grad psi, p += psi (the FP64 residual runs at evp_sync)
    K_LEVELSET,       // S9: TVD-RK3 stage of level-set advection or re-distancing
    K_INTERFACE,      // S9: H, normals, curvature, CSF and buoyancy force
    K_IBM,            // discrete-forcing IBM of rigid particles (multi-direct iterations)
    K_COUNT
};

// Geometry as seen by the kernels.  Spacings are passed as reciprocals.
template <typename T>
struct Geo {
    int nx, ny, nz, walls;
    T idx, idy, idz;      // 1/dx, 1/dy, 1/dz
};

// ----------------------------------------------------------------- index maps
__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ size_t lin(const Geo<T>& g, int i, int j, int k) {
    return ((size_t)k * g.ny + j) * g.nx + i;
}

// y index of a cell-centred value: zero-gradient copy at walls, periodic wrap otherwise
template <typename T>
__device__ __forceinline__ int ycen(const Geo<T>& g, int j) {
    if (g.walls) return j < 0 ? 0 : (j >= g.ny ? g.ny - 1 : j);
    return wrap(j, g.ny);
}

// u or w (centred in y) at (i, j, k) with i, k wrapped and the no-slip odd ghost in y
template <typename T>
__device__ __forceinline__ T ld_uw(const Geo<T>& g, const T* __restrict__ F, int i, int j, int k) {
    i = wrap(i, g.nx);
    k = wrap(k, g.nz);
    if (g.walls) {
        if (j < 0) return -__ldg(F + lin(g, i, -1 - j, k));
        if (j >= g.ny) return -__ldg(F + lin(g, i, 2 * g.ny - 1 - j, k));
        return __ldg(F + lin(g, i, j, k));
    }
    return __ldg(F + lin(g, i, wrap(j, g.ny), k));
}

// v (on y faces) at (i, j, k): zero outside the stored range at walls
template <typename T>
__device__ __forceinline__ T ld_v(const Geo<T>& g, const T* __restrict__ F, int i, int j, int k) {
    i = wrap(i, g.nx);
    k = wrap(k, g.nz);
    if (g.walls) {
        if (j < 0 || j >= g.ny) return T(0);
        return __ldg(F + lin(g, i, j, k));
    }
    return __ldg(F + lin(g, i, wrap(j, g.ny), k));
}

// centred scalar at (i, j, k)
template <typename T>
__device__ __forceinline__ T ld_c(const Geo<T>& g, const T* __restrict__ F, int i, int j, int k) {
    return __ldg(F + lin(g, wrap(i, g.nx), ycen(g, j), wrap(k, g.nz)));
}

// ------------------------------------------------------------- model constants
struct ModelConst {
    int model;          // evp_model
    double inv_lam;     // 1/lambda
    double gmod;        // mu_p / lambda
    double tau_y;       // Saramito yield stress
    double L2, a_fene;  // FENE-P L^2 and a = L^2/(L^2-3)
    double mu_s;        // solvent viscosity
    double art_diff;    // local artificial diffusivity of B (0: off)
    // the same constants rounded to single precision on the host (set_single)
    float f_inv_lam, f_gmod, f_tau_y, f_L2, f_a_fene, f_mu_s, f_art_diff;
    void set_single() {
        f_inv_lam = float(inv_lam);
        f_gmod = float(gmod);
        f_tau_y = float(tau_y);
        f_L2 = float(L2);
        f_a_fene = float(a_fene);
        f_mu_s = float(mu_s);
        f_art_diff = float(art_diff);
    }
};

// A model constant in the kernel's precision T: single-precision kernels read the
// host-rounded copy, so that no kernel converts a double (on GB300 a conversion
// instruction runs on the narrow FP64 pipe, and the compiler may recompute such a
// conversion inside a loop rather than keep it in a register).
template <typename T>
__device__ __forceinline__ T kconst(double d, float f) {
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}

// Conversions between binary32 and binary64 (IEEE 754) done branch-free with
// integer operations, so that FP64 work on FP32 data leaves the (narrow) FP64 pipe
// to the arithmetic and keeps batched loads free to be scheduled early.  They give
// the conversion instruction's result bit for bit for every normal number, zero
// and infinity; values in the binary32 subnormal range (magnitude below 2^-126)
// become a signed zero on both sides of the conversion (an absolute difference
// below 1.2e-38), and a NaN stays a NaN.

// binary32 -> binary64: the exponent is rebiased by 1023 - 127 = 896 and the
// 23-bit fraction moves to the top of the 52-bit one; exponent field 0 gives a
// signed zero, exponent field 255 (infinity, NaN) stays all ones.
__device__ __forceinline__ double widen_f32(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned sign = b & 0x80000000u;
    const unsigned E = e == 0xffu ? 0x7ffu : e + 896u;
    const unsigned hi = e ? (sign | (E << 20) | ((b & 0x7fffffu) >> 3)) : sign;
    const unsigned lo = e ? (b << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen_f32(double x) { return x; }

// binary64 -> binary32, rounding to nearest with ties to even.  Where the result
// is a normal float (biased exponent 897..1150 of x) the 29 dropped fraction bits
// decide the increment, and a carry out of the fraction moves into the exponent
// (up to infinity, as rounding to nearest does).  Magnitudes below 2^-126 give a
// signed zero, larger exponents infinity, and a NaN gives the quiet NaN.
__device__ __forceinline__ float narrow_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned sign = hi & 0x80000000u;
    const unsigned keep = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | lo);
    unsigned r = sign + ((e - 896u) << 23) + keep + up;
    r = e < 897u ? sign : r;
    r = e > 1150u ? (sign | 0x7f800000u) : r;
    r = nan ? (sign | 0x7fc00000u) : r;
    return __uint_as_float(r);
}
__device__ __forceinline__ float narrow_to(double x, float*) { return narrow_f64(x); }
__device__ __forceinline__ double narrow_to(double x, double*) { return x; }

// ------------------------------------------------------------ argument blocks
template <typename T>
struct StressArgs {
    const T* U;
    const T* V;
    const T* W;
    const T* B[6];
    T* Bn[6];          // B^k (update mode)
    T* RT[6];          // history RT^{k-2} in / RT^{k-1} out (update), or RT out (rhs mode)
    T dt_zeta, dt_xi;
    int read_hist, write_hist, rhs_only;
    unsigned* status;
    const T* H;        // two-phase: Heaviside of the level set (null: single phase)
    T mu_p1, mu_p2;    // two-phase: polymer viscosity of fluid 1 (H = 1) and fluid 2
    // update modes: summed polymer stress tau(B^k) + tau(B^{k-1}) out for the
    // momentum step (Table 1 with the state's G); null: not written
    T* S[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

template <typename T>
struct MomentumArgs {
    const T* U;
    const T* V;
    const T* W;
    const T* P;
    const T* Bo[6];    // B^{k-1}
    const T* Bn[6];    // B^k
    T* Us;
    T* Vs;
    T* Ws;             // u* out
    T* NH[3];          // history N^{k-2} in / N^{k-1} out
    T dt, zeta, xi, alpha;
    int read_hist, write_hist, has_stress;
    T dpdx, abc_amp;
    int cn = 0;        // implicit viscous option: N without the viscous term, alpha mu lap(u) explicit
    const T* phis_o = nullptr;   // soft particles: solid fraction at levels k-1 and k,
    const T* phis_n = nullptr;   //   tau = phi_s G (B - I) (neo-Hookean model)
    const T* trig;     // ABC force tables: sin/cos of k x_i, k y_j, k z_k (6 arrays)
    const T* solid[3]; // volume penalisation: solid fractions at u, v, w nodes (null: off)
    // summed polymer stress tau^k + tau^{k-1} written by the stress kernel; null:
    // built here from Bo and Bn
    const T* S[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    unsigned* status = nullptr;  // the state's status word (reports of the bounds-checked build)
};

template <typename T>
struct FFTTables {
    const typename Cplx<T>::type* twx;   // exp(-2 pi i m / nx), m < nx
    const typename Cplx<T>::type* twy;
    const typename Cplx<T>::type* twz;
    int radx[12], nrx;
    int rady[12], nry;
    int radz[12], nrz;
    const T* lamx;     // modal eigenvalues (2 - 2cos(2 pi m/n))/h^2, T precision
    const T* lamy;
    const T* lamz;
    const double2* thomas_m;  // walls: (m_j, c'_j) per system, [nz/2+1][ny][nxh]
    int thomas_ds = 0;        // single precision: the table (and the Helmholtz tables) in the
                              // double-single format of thomas_table_ds, swept so
    double idy2;              // walls: 1/dy^2 in FP64 (the Thomas sub-diagonal)
};

template <typename T>
struct PoissonArgs {
    // right-hand side: either divergence of (Us, Vs, Ws) times rscale, or a given field
    const T* Us;
    const T* Vs;
    const T* Ws;
    const T* rhs;      // if non-null, used instead of the divergence
    T rscale;
    typename Cplx<T>::type* spec;     // [nz][ny][nxh] complex
    T* psi;            // psi out
    // Helmholtz problems x - c lap(x) = r (implicit viscous option): with walls the
    // Thomas table and constant sub-diagonal replace the Poisson ones (no pinned
    // mode); periodic y divides the modes by 1 + hcoef lam.  ttab null: Poisson.
    const double2* ttab = nullptr;
    double tsub = 0.0;
    T hcoef = T(0);
    double norm;       // 1/(nx nz) (walls) or 1/(nx ny nz) (periodic)
    T out_scale;       // factor applied to psi by the inverse x pass (walls: norm)
    double* scratch;   // walls: FP64 forward-sweep values, 2 (nx/2+1) ny nz doubles
};

template <typename T>
struct CorrectArgs {
    const T* Us;
    const T* Vs;
    const T* Ws;
    const T* psi;
    T* U;
    T* V;
    T* W;
    T* P;              // p += psi if non-null (p = psi with p_replace)
    int p_replace;     // AB2 step: the pressure is psi itself (Eq. projection)
    T coef;            // 2 alpha dt (or 1 for a plain projection)
    unsigned* status;
};

// two-phase step (level set, interface force, AB2 momentum)
template <typename T>
struct LsArgs {
    const T* U;
    const T* V;
    const T* W;        // velocity u^n (advection)
    const T* phin;     // phi at the start of the TVD-RK3 step (pointwise term)
    const T* phis;     // stage input (stencil)
    const T* phi0;     // re-distancing: phi before it started, for S(phi0)
    T* out;            // out = pt_a phin + pt_b (phis + dt rhs(phis))
    T pt_a, pt_b, dt;
    T h;               // grid spacing (S(phi0) smoothing width)
};

template <typename T>
struct IfaceArgs {
    const T* phi;
    T* H;
    T* n[3];           // unit normal at centres
    T* f[3];           // interface force at centres
    double* partials;  // per-block sums of 1 - H
    double* mean_1mH;  // domain mean of 1 - H
    T eps, sigma, drho_g;
};

// soft particles: RK3 update of the solid fraction, phi^k = phi^{k-1} + dt (zeta R
// + xi R_hist) with R = -u^{k-1}.grad phi^{k-1} (WENO5)
template <typename T>
struct PhisArgs {
    const T* U;
    const T* V;
    const T* W;
    const T* phi;      // level k-1
    T* phin;           // level k
    T* hist;           // R of the previous substep (in / out)
    T dt_zeta, dt_xi;
    int read_hist, write_hist;
};

// discrete-forcing IBM of rigid particles (k_ibm.cu); Lagrangian points of
// particle p are l = start[p] .. start[p+1]-1
template <typename T>
struct IbmArgs {
    T* U[3];                // u* -> u** in place
    const double* off;      // [nl][3] point offsets from the particle centre
    const int* owner;       // [nl] particle of each point
    const int* start;       // [np+1]
    const double* dvl;      // [np] volume carried by each point of the particle
    double* centre;         // [np][3] (advanced by the finishing kernel)
    const double* pvel;     // [np][3] prescribed velocity
    const double* pomg;     // [np][3] prescribed angular velocity
    double* Facc;           // [nl][3] accumulated Lagrangian force
    double* dF;             // [nl][3] this iteration's increment
    double* pforce;         // [np][6] force and torque on each particle
    double* pvel_w;         // [np][3] velocity, updated for free particles
    double* pomg_w;         // [np][3] angular velocity, updated for free particles
    const double* prad;     // [np] radius
    const double* pdens;    // [np] density ratio rho_p / rho_f (0: prescribed motion)
    double* I0;             // [np][6] inner-fluid integrals int u dV, int r x u dV before the forcing
    double* I1;             // [np][6] ... after it
    int nl, np, nx, ny, nz, walls, any_free;
    double dx, dy, dz, y0;  // cell sizes, y of the bottom of the box
    double lx, ly, lz;
    double dts;             // the substep's time increment 2 alpha dt
    double gravity;         // along -y, acting on free particles
};

// mass-preserving level-set shift (two-phase step): phi <- phi + d with d from
// Newton iterations on the smoothed drop volume
template <typename T>
struct MassArgs {
    T* phi;
    T eps;
    double* partials;  // per-block sums: [0, np) of 1 - H(phi + d), [np, 2 np) of delta(phi + d)
    double* v0;        // target drop volume
    double* d;         // accumulated shift
    double dv;         // cell volume
};

template <typename T>
struct MomAB2Args {
    const T* U;
    const T* V;
    const T* W;
    const T* B[6];     // B^n
    const T* H;
    const T* f[3];     // interface force at centres
    T* Us;
    T* Vs;
    T* Ws;
    T* NH[3];          // RU^{n-1} in (if read_hist), RU^n out
    T w1dt, w0dt;      // dt * 3/2 and dt * (-1/2) (dt and 0 on the first step)
    int read_hist;
    T mu_s1, mu_s2, mu_p1, mu_p2, inv_lam, L2, a_fene;
    // density contrast (rho_ratio > 0): rho = H + rho_ratio (1 - H), gravity along -y
    T rho_ratio, gravity;
    const double* mean_1mH;   // domain mean of 1 - H (for the mean density)
};

// Dong-Shen split projection (Eqs. poisson-LS, projection-LS)
template <typename T>
struct SplitArgs {
    const T* Us;
    const T* Vs;
    const T* Ws;       // u*
    const T* P;        // p^n
    const T* Pold;     // p^{n-1}
    const T* H;        // Heaviside at n+1
    T* R;              // right-hand side out (rhs kernel) / p^{n+1} in (correction)
    T* U;
    T* V;
    T* W;              // u^{n+1} out
    T rho_ratio, rho0, dt;
    unsigned* status;
};

// ------------------------------------------------------------------- batches
// A batch advances several states with one launch per kernel phase.  The members'
// argument blocks travel in the kernel's parameter space (at most 32 KB), so a
// launch holds at most EVP_BATCH_MAX members.
constexpr int EVP_BATCH_MAX = 64;

template <typename T>
struct StressMember {
    Geo<T> g;
    ModelConst mc;
    StressArgs<T> a;
    int kz;            // z planes per work item
};
template <typename T>
struct StressBatch {
    StressMember<T> m[EVP_BATCH_MAX];
};

template <typename T>
struct MomentumMember {
    Geo<T> g;
    ModelConst mc;
    MomentumArgs<T> a;
    int kz;
};
template <typename T>
struct MomentumBatch {
    MomentumMember<T> m[EVP_BATCH_MAX];
};

// Poisson passes and correction of members that share one grid (the FFT kernels
// are specialised by length): member = blockIdx.z of the launch
template <typename T>
struct PoissonBatch {
    PoissonArgs<T> a[EVP_BATCH_MAX];
};
template <typename T>
struct CorrectBatch {
    CorrectArgs<T> a[EVP_BATCH_MAX];
};

// ----------------------------------------------------------- launch functions
// Each returns cudaSuccess or the launch error; ``t`` is a timing hook that
// records events around the launch when enabled.
struct TimingHook {
    void (*begin)(void* ctx, int kid);
    void (*end)(void* ctx, int kid);
    void* ctx;
    bool pdl = false;    // launch with programmatic dependent launch (see launch_k)
    void b(int kid) const { if (begin) begin(ctx, kid); }
    void e(int kid) const { if (end) end(ctx, kid); }
};

// Programmatic dependent launch.  A kernel launched with ``pdl`` may be scheduled
// while the previous kernel on the stream is still running (its launch and
// set-up overlap that kernel's tail); every such kernel first executes pdl_wait(),
// which returns once the previous grid has completed and its memory is visible,
// before it touches global memory.  pdl_trigger() lets the next kernel be
// scheduled once every CTA of this grid has started.  Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ---- bounds-checked build (compiled with -DEVP_DEBUG into libevp_debug.so)
// The stencil kernels check every staged copy: its source inside one of the
// kernel's fields, its shared-memory destination inside the kernel's staging
// area, 16-byte alignment of both for 16-byte copies.  A failed check skips the
// copy and sets a per-thread flag, which the kernel ORs into its status word as
// EVP_BIT_BOUNDS when it ends (evp_sync then returns EVP_ERR_BOUNDS); nothing
// traps.  The staging area is filled with NaN bytes before a tile starts, so a
// stencil that reads a value no copy has written makes its output non-finite.
// Without EVP_DEBUG the checks compile to nothing.
#ifdef EVP_DEBUG
#define EVP_DBG_DECL bool dbg_fail_ = false
#define EVP_DBG_OK(cond) ((cond) || (dbg_fail_ = true, false))
#define EVP_DBG_REPORT(status)                                          \
    do {                                                                \
        if (dbg_fail_ && (status)) atomicOr((status), EVP_BIT_BOUNDS);  \
    } while (0)
// a staged copy of n elements from s (global) to d (shared); v16: a 16-byte copy.
// The tile function defines dbg_src_ok(p, n) and dbg_dst_ok(p, n) for its fields
// and its staging area.
#define EVP_STAGE_OK(d, s, n, v16) \
    EVP_DBG_OK(dbg_src_ok((s), (n)) && dbg_dst_ok((d), (n)) && (!(v16) || (dbg_aligned16(s) && dbg_aligned16(d))))
#else
#define EVP_DBG_DECL [[maybe_unused]] constexpr bool dbg_fail_ = false
#define EVP_DBG_OK(cond) true
#define EVP_STAGE_OK(d, s, n, v16) true
#define EVP_DBG_REPORT(status) \
    do {                       \
    } while (0)
#endif

// [p, p + n) inside [base, base + count) (debug checks)
template <typename T>
__device__ __forceinline__ bool dbg_within(const T* p, int n, const T* base, size_t count) {
    return base != nullptr && p >= base && p + n <= base + count;
}
__device__ __forceinline__ bool dbg_aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Fill [smem, smem + bytes) with 0xff bytes (a NaN in binary32 and binary64);
// bytes a multiple of 16 and smem 16-byte aligned.  Ends with a barrier.
__device__ __forceinline__ void dbg_poison(unsigned char* smem, size_t bytes) {
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    uint4* p = reinterpret_cast<uint4*>(smem);
    for (size_t q = t; q < bytes / 16; q += nt) p[q] = make_uint4(~0u, ~0u, ~0u, ~0u);
    __syncthreads();
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Host: the FP64 Thomas table for the wall-bounded Poisson solve.  For every
// (kz <= nz/2, kx) system of size ny (rows idy2 psi_{j-1} - (2 idy2 + lx + lz)
// psi_j + idy2 psi_{j+1}, Neumann rows at both ends, the (0, 0) system pinned by
// psi_0 = 0) entry j holds (m_j, c'_j): the reciprocal pivot m_j = 1/(b_j - a_j c'_{j-1})
// and the normalised super-diagonal c'_j = u_j m_j (0 on the last and the pinned
// row).  Layout [kz][j][kx] as interleaved (m, c') pairs.
inline std::vector<double> thomas_table(int ny, int nz, int nxh, double dy, const std::vector<double>& lamx,
                                        const std::vector<double>& lamz_half) {
    const int nkz = nz / 2 + 1;
    const double idy2 = 1.0 / (dy * dy);
    std::vector<double> M((size_t)nkz * ny * nxh * 2);
    for (int kz = 0; kz < nkz; ++kz)
        for (int kx = 0; kx < nxh; ++kx) {
            const double lm = lamx[kx] + lamz_half[kz];
            const bool pinned = (kx == 0 && kz == 0);
            double cprev = 0.0;
            for (int j = 0; j < ny; ++j) {
                const double lo = j > 0 ? idy2 : 0.0;
                double up = j < ny - 1 ? idy2 : 0.0;
                double d = -2.0 * idy2 - lm + (j == 0 ? idy2 : 0.0) + (j == ny - 1 ? idy2 : 0.0);
                if (pinned && j == 0) {
                    d = 1.0;
                    up = 0.0;
                }
                const double m = 1.0 / (d - lo * cprev);
                cprev = up * m;
                const size_t o = 2 * (((size_t)kz * ny + j) * nxh + kx);
                M[o] = m;
                M[o + 1] = cprev;
            }
        }
    return M;
}

// Host: FP64 Thomas table (m_j, c'_j), same layout as thomas_table, of the
// Helmholtz systems x - c lap(x) = r of the implicit viscous option per
// (kz <= nz/2, kx): rows -cy x_{j-1} + (1 + c(lx + lz) + 2 cy) x_j - cy x_{j+1},
// cy = c/dy^2.  kind_v false (u, w centred in y): the odd no-slip mirror adds cy
// to the first and last diagonals.  kind_v true (v on y-faces): rows 0..ny-2
// with zero Dirichlet faces beyond them; row ny-1 (the top wall face) has m = 0,
// which makes its solution zero.
inline std::vector<double> helmholtz_table(int ny, int nz, int nxh, double dy, const std::vector<double>& lamx,
                                           const std::vector<double>& lamz_half, double c, bool kind_v) {
    const int nkz = nz / 2 + 1;
    const double cy = c / (dy * dy);
    const int m_rows = kind_v ? ny - 1 : ny;
    std::vector<double> M((size_t)nkz * ny * nxh * 2, 0.0);
    for (int kz = 0; kz < nkz; ++kz)
        for (int kx = 0; kx < nxh; ++kx) {
            const double base = 1.0 + c * (lamx[kx] + lamz_half[kz]) + 2.0 * cy;
            double cprev = 0.0;
            for (int j = 0; j < m_rows; ++j) {
                const double lo = j > 0 ? -cy : 0.0;
                const double up = j < m_rows - 1 ? -cy : 0.0;
                double d = base;
                if (!kind_v && (j == 0 || j == m_rows - 1)) d += cy;
                const double m = 1.0 / (d - lo * cprev);
                cprev = up * m;
                const size_t o = 2 * (((size_t)kz * ny + j) * nxh + kx);
                M[o] = m;
                M[o + 1] = cprev;
            }
        }
    return M;
}

// Host: a Thomas table (pairs (m_j, c'_j) of doubles) in the format of the
// single-precision states, whose sweep runs in double-single arithmetic: every
// double x becomes the unevaluated sum hi + lo of two floats, hi = x rounded to
// float and lo = the remainder x - hi rounded to float, so an entry is the four
// floats (m_hi, m_lo, c'_hi, c'_lo) in the 16 bytes of the double pair.
inline std::vector<float> thomas_table_ds(const std::vector<double>& M) {
    std::vector<float> F(M.size() * 2);
    for (size_t q = 0; q < M.size(); ++q) {
        const float hi = static_cast<float>(M[q]);
        F[2 * q] = hi;
        F[2 * q + 1] = static_cast<float>(M[q] - static_cast<double>(hi));
    }
    return F;
}

// device self-test of widen_f32 / narrow_f64 (k_selftest.cu)
cudaError_t run_selftest(unsigned long long* mismatches);
// best rate of plain FMAs of the current device, in FLOP/s (k_selftest.cu)
cudaError_t run_fma_peak(int precision, double* flops);

template <typename T>
cudaError_t launch_stress(const Geo<T>& g, const ModelConst& mc, const StressArgs<T>& a,
                          cudaStream_t st, const TimingHook& th);

template <typename T>
cudaError_t launch_momentum(const Geo<T>& g, const ModelConst& mc, const MomentumArgs<T>& a,
                            cudaStream_t st, const TimingHook& th);

// Batched launches.  work: device list of int4 (member, tile x, tile y, z chunk);
// ctas: size of the persistent grid.  The stress batch holds members of one model
// and one staging kind (vec: nx * sizeof(T) % 16 == 0); mode 1, 2, 3 as the
// update modes of the stress kernel.  The momentum batch reads the summed stress.
template <typename T>
cudaError_t launch_stress_batch(const StressBatch<T>& p, int model, int mode, bool vec, const int4* work, int nwork,
                                int ctas, cudaStream_t st);
template <typename T>
cudaError_t launch_momentum_batch(const MomentumBatch<T>& p, bool vec, const int4* work, int nwork, int ctas,
                                  cudaStream_t st);
// tiles and resident CTAs per SM of the z-marching kernels
int stress_tile_x();
int stress_tile_y();
int momentum_tile_x();
int momentum_tile_y();
template <typename T>
int stress_ctas_per_sm();
template <typename T>
int momentum_ctas_per_sm();
// Poisson solve (divergence of u* as right-hand side) and correction of n members
// that share grid g and tables tb; tk: kx columns per block of the column passes
template <typename T>
cudaError_t launch_poisson_batch(const Geo<T>& g, const FFTTables<T>& tb, const PoissonBatch<T>& p, int n, int tk,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_correct_batch(const Geo<T>& g, const CorrectBatch<T>& p, int n, cudaStream_t st);

template <typename T>
cudaError_t launch_poisson(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a,
                           cudaStream_t st, const TimingHook& th);

template <typename T>
cudaError_t launch_correct(const Geo<T>& g, const CorrectArgs<T>& a, cudaStream_t st,
                           const TimingHook& th);
// FP64 max |div u| of the stored velocity (U, V, W) into *maxdiv (bits of a
// non-negative double, atomic max: the caller zeroes it); non-finite -> status
template <typename T>
cudaError_t launch_div_residual(const Geo<T>& g, const T* U, const T* V, const T* W, double idx, double idy,
                                double idz, unsigned long long* maxdiv, unsigned* status, cudaStream_t st);

// ---- monitoring reductions (evp_diagnostics)
constexpr int DIAG_BLOCKS = 8 * 152;   // at most this many block partials
struct DiagPart {
    double ke;                     // sum of u^2 + v^2 + w^2 (not yet scaled by dx dy dz / 2)
    double min_det, max_tr;        // of B over the cells
    unsigned long long yielded;    // cells with F > 0
    unsigned long long nonfinite;  // cells with a NaN or infinite value
};
template <typename T>
struct DiagArgs {
    const T* U;
    const T* V;
    const T* W;
    const T* B[6];     // null: no conformation (Newtonian)
    const T* H;        // Saramito two-phase: Heaviside, tau = (mp1 H / lambda)(B - I); null: single phase
    double gm;         // single phase: mu_p / lambda
    double mp1, inv_lam;
    double tau_y;
    int yield_mode;    // 0: no yield surface, 1: every cell flows, 2: Saramito |tau^d| > tau_y
};
// two launches on st: block partials into parts[0 .. DIAG_BLOCKS), their fold into *out
template <typename T>
cudaError_t launch_diag(const Geo<T>& g, const DiagArgs<T>& a, DiagPart* parts, DiagPart* out, cudaStream_t st);

template <typename T>
cudaError_t launch_ls_stage(const Geo<T>& g, const LsArgs<T>& a, bool reinit, cudaStream_t st,
                            const TimingHook& th);

template <typename T>
size_t iface_partials(const Geo<T>& g);

template <typename T>
cudaError_t launch_interface(const Geo<T>& g, const IfaceArgs<T>& a, cudaStream_t st, const TimingHook& th);

// the whole particle coupling of one substep: inner integrals of u^{k-1} (free
// particles), the multi-direct forcing of u* (in a.U), force and torque, inner
// integrals of u**, particle update
template <typename T>
cudaError_t launch_phis(const Geo<T>& g, const PhisArgs<T>& a, cudaStream_t st, const TimingHook& th);

template <typename T>
cudaError_t launch_ibm(const IbmArgs<T>& a, const T* const uold[3], int iters, cudaStream_t st,
                       const TimingHook& th);

// mode 0: v0 <- drop volume of phi; mode 1: ``iters`` Newton updates of d, then phi += d
template <typename T>
cudaError_t launch_mass_correct(const Geo<T>& g, const MassArgs<T>& a, int mode, int iters, cudaStream_t st,
                                const TimingHook& th);

template <typename T>
cudaError_t launch_momentum_ab2(const Geo<T>& g, int model, const MomAB2Args<T>& a, cudaStream_t st,
                                const TimingHook& th);

template <typename T>
cudaError_t launch_split_rhs(const Geo<T>& g, const SplitArgs<T>& a, cudaStream_t st, const TimingHook& th);

template <typename T>
cudaError_t launch_split_correct(const Geo<T>& g, const SplitArgs<T>& a, cudaStream_t st, const TimingHook& th);

// radix plan of n = 4^a 3^b 2^c (radix-4 first); returns the number of stages or -1
int fft_radices(int n, int* rad);

}  // namespace evp
