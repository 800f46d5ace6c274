// S3: momentum predictor of Eqs. NS-num1 and rk3 on the staggered grid.
//
// u* = u^{k-1} + dt [zeta^k N^{k-1} + xi^k N^{k-2} - 2 alpha^k grad p^{k-1}
//                    + alpha^k div(tau^k + tau^{k-1})]
// N  = -div(uu) + mu_s lap(u) + f
//
// div(uu) by second-order central differences (products at centres and edges),
// the viscous term explicit with the advective weights, div(tau) at faces from
// centre tau with 4-point edge averages for the off-diagonal parts (div is linear,
// so the two stress levels are summed first).  Each thread computes the three
// faces (i+1/2, j, k), (i, j+1/2, k), (i, j, k+1/2) of its cell; with walls the
// top y-face stays zero.
//
// A 32 x 4 tile walks a chunk of z planes.  Shared memory holds planes k-1..k+1
// (1-cell x-y halo) of u, v, w and p, and of the summed stress S = tau^k + tau^{k-1},
// plus the cell's momentum history; planes are staged two ahead by cp.async.  S is
// either written by the stress kernel and staged like the velocity (5-slot rings,
// one barrier per plane) or built here from the staged raw B^{k-1} and B^k planes
// (3-slot ring, a build phase between two barriers).  A plane row is 40 wide
// with the tile's interior at columns 4..35, so that when nx is a multiple of
// 16 bytes' worth of elements every row is staged in 16-byte cp.async chunks
// (x = i0-4 .. i0+35, wrapped periodically chunk by chunk); other grids stage
// element by element.
#include <type_traits>

#include "evp_internal.cuh"

namespace evp {

namespace {

constexpr int TX = 32, TY = 4, NT = TX * TY;
constexpr int VW = TX + 8, XO = 4;                       // plane row width; column of the tile's i0
constexpr int VH = TY + 2, VPL = VW * VH;                // rows j0-1 .. j0+TY
constexpr int SW = TX + 2;                               // columns the stencils use: XO-1 .. XO+TX
constexpr int NV = (SW * VH + NT - 1) / NT;              // used plane cells per thread (2)

template <typename T>
__device__ __forceinline__ T sq(T x) { return x * x; }

__device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}
// a in [-n, 2n): one conditional wrap, no division
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// 16-byte asynchronous copy (L2 only)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// all but the most recently committed group have landed
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Planes are staged two ahead (the forms that build the summed stress here, and the
// batched kernel): while plane k is computed, plane k+2 has landed (or is landing)
// and plane k+3 is being requested.
template <typename T>
struct MomSmem {
    T V[3][5][VPL];      // u, v, w: ring slots for planes k-1 .. k+3
    T S[6][3][VPL];      // summed stress: ring slots for planes k-1 .. k+1
    T Braw[2][12][VPL];  // raw B^{k-1} (0..5) and B^k (6..11) of planes k+2 and k+3
    T P[4][VPL];         // pressure planes k .. k+3
    T H[4][3][NT];       // momentum history of the tile's cells, planes k .. k+2
};
// The summed stress written by the stress kernel is staged like the velocity:
// ring slots for planes k-1 .. k+3, no raw B and no build phase.
template <typename T>
struct MomSmemS {
    T V[3][5][VPL];
    T S[6][5][VPL];
    T P[4][VPL];
    T H[4][3][NT];
};
// Staged one plane ahead (D1): while plane k is computed, plane k+2 is being
// requested; fewer slots, so six CTAs fit on an SM in FP32.  Of the summed
// stress only xz and yz are read at planes k-1 and k+1 (the z derivatives and
// edge averages of div tau); xx, xy, yy and zz are read at planes k (and k+1 for
// zz) and keep three slots.
template <typename T>
struct MomSmemS1 {
    T V[3][4][VPL];      // planes k-1 .. k+2
    T S4[2][4][VPL];     // S_xz, S_yz: planes k-1 .. k+2
    T S3[4][3][VPL];     // S_xx, S_xy, S_yy, S_zz: planes k .. k+2
    T P[3][VPL];         // planes k .. k+2
    T H[2][3][NT];       // planes k, k+1
};
template <typename T, bool SPRE, bool D1>
using MomSmemOf = std::conditional_t<SPRE, std::conditional_t<D1, MomSmemS1<T>, MomSmemS<T>>, MomSmem<T>>;
// ring slots of velocity / stress, pressure and history planes (kk >= -1)
template <bool D1>
__device__ __forceinline__ int vs_of(int kk) { return D1 ? (kk + 4) % 4 : (kk + 5) % 5; }
template <bool D1>
__device__ __forceinline__ int ps_of(int kk) { return D1 ? (kk + 3) % 3 : (kk & 3); }
template <bool D1>
__device__ __forceinline__ int hs_of(int kk) { return D1 ? (kk & 1) : (kk & 3); }

// VEC: rows are staged in 16-byte chunks (needs nx * sizeof(T) % 16 == 0)
// SPRE: the summed stress comes precomputed (MomentumArgs::S); MODEL is then unused
// One tile: the 32 x 4 columns (bx, by) over the z chunk bz of kz_chunk planes.
template <typename T, int MODEL, bool VEC, bool SPRE, bool D1 = false>
__device__ __forceinline__ void momentum_tile(const Geo<T>& g, const ModelConst& mc, const MomentumArgs<T>& a,
                                              int kz_chunk, int bx, int by, int bz, unsigned char* smraw) {
    static_assert(!D1 || SPRE, "one-ahead staging is a form of the precomputed-stress kernel");
    MomSmemOf<T, SPRE, D1>& sm = *reinterpret_cast<MomSmemOf<T, SPRE, D1>*>(smraw);
    EVP_DBG_DECL;
#ifdef EVP_DEBUG
    dbg_poison(smraw, sizeof(MomSmemOf<T, SPRE, D1>));
    const size_t dbg_n = (size_t)g.nx * g.ny * g.nz;
    auto dbg_src_ok = [&](const T* p, int n) {
        if (dbg_within(p, n, a.U, dbg_n) || dbg_within(p, n, a.V, dbg_n) || dbg_within(p, n, a.W, dbg_n) ||
            dbg_within(p, n, a.P, dbg_n) || dbg_within(p, n, a.phis_o, dbg_n) || dbg_within(p, n, a.phis_n, dbg_n))
            return true;
        for (int c = 0; c < 6; ++c)
            if (dbg_within(p, n, a.Bo[c], dbg_n) || dbg_within(p, n, a.Bn[c], dbg_n) || dbg_within(p, n, a.S[c], dbg_n))
                return true;
        for (int q = 0; q < 3; ++q)
            if (dbg_within(p, n, (const T*)a.NH[q], dbg_n) || dbg_within(p, n, a.solid[q], dbg_n)) return true;
        return false;
    };
    auto dbg_dst_ok = [&](const T* d, int n) {
        return (const unsigned char*)d >= smraw &&
               (const unsigned char*)(d + n) <= smraw + sizeof(MomSmemOf<T, SPRE, D1>);
    };
#endif
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = bx * TX, j0 = by * TY;
    const int k0 = bz * kz_chunk, k1 = min(k0 + kz_chunk, g.nz);
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < g.nx && j < g.ny;
    const size_t plane = (size_t)g.nx * g.ny;
    const bool stress = MODEL != EVP_NEWTONIAN;

    // Row ghost rules (walls): centred fields copy the nearest row; u and w take
    // the odd mirror (no slip), v is zero outside the stored faces.  Periodic y
    // wraps.  For plane row y (= j0-1+r) returns the source row and the factor
    // (+1 copy, -1 negated copy, 0 zero) of velocity component q, or of a centred
    // field for q = 3.
    auto row_rule = [&](int gy, int q, int& src) -> int {
        if (!g.walls) {
            src = pmod(gy, g.ny);
            return 1;
        }
        if (q == 3) {
            src = min(max(gy, 0), g.ny - 1);
            return 1;
        }
        const bool inside = gy >= 0 && gy < g.ny;
        if (q == 1) {
            src = inside ? gy : 0;
            return inside ? 1 : 0;
        }
        const int my = gy < 0 ? -1 - gy : (gy >= g.ny ? 2 * g.ny - 1 - gy : gy);
        src = min(max(my, 0), g.ny - 1);
        return (my >= 0 && my < g.ny) ? (inside ? 1 : -1) : 0;
    };

    // element-wise staging: this thread's used plane cells (row r, column XO-1+c)
    size_t coff[NV], voff[3][NV];
    signed char vfac[3][NV];
    int psm[NV];
    // chunk staging: this thread's 16-byte chunk of a plane (row ch / CPR)
    constexpr int E = 16 / (int)sizeof(T);                // elements per chunk
    constexpr int CPR = VW / E, NCH = CPR * VH;           // chunks per row / plane
    int csm = -1;
    size_t ccoff = 0, cvoff[3] = {0, 0, 0};
    signed char cvfac[3] = {0, 0, 0};
    if (VEC) {
        if (tid < NCH) {
            const int r = tid / CPR, q0 = (tid - r * CPR) * E;
            csm = r * VW + q0;
            const int gx = pmod(i0 - XO + q0, g.nx);      // a whole chunk: nx is a multiple of E
            int src;
            row_rule(j0 - 1 + r, 3, src);
            ccoff = (size_t)src * g.nx + gx;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                cvfac[q] = (signed char)row_rule(j0 - 1 + r, q, src);
                cvoff[q] = (size_t)src * g.nx + gx;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NV; ++r) {
        const int e = tid + r * NT;
        const int vy = e / SW, vx = e - vy * SW;
        psm[r] = e < SW * VH ? vy * VW + vx + XO - 1 : -1;
        coff[r] = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            voff[q][r] = 0;
            vfac[q][r] = 0;
        }
        if (e >= SW * VH) continue;
        const int gx = pmod(i0 + vx - 1, g.nx);
        int src;
        row_rule(j0 + vy - 1, 3, src);
        coff[r] = (size_t)src * g.nx + gx;        // also the soft particles' solid-fraction reads
        if constexpr (!VEC) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                vfac[q][r] = (signed char)row_rule(j0 + vy - 1, q, src);
                voff[q][r] = (size_t)src * g.nx + gx;
            }
        }
    }
    const T* vel[3] = {a.U, a.V, a.W};
    // E elements from global (one 16-byte vector) into shared, times fac (+1, -1, 0)
    auto copy_scaled = [&](T* dst, const T* src, int fac) {
        if (sizeof(T) == 4) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (fac) {
                v = __ldg(reinterpret_cast<const float4*>(src));
                v.x = -v.x; v.y = -v.y; v.z = -v.z; v.w = -v.w;
            }
            *reinterpret_cast<float4*>(dst) = v;
        } else {
            double2 v = make_double2(0.0, 0.0);
            if (fac) {
                v = __ldg(reinterpret_cast<const double2*>(src));
                v.x = -v.x; v.y = -v.y;
            }
            *reinterpret_cast<double2*>(dst) = v;
        }
    };
    auto fetch_vel = [&](int kk) {
        const size_t pv = (size_t)wrap1(kk, g.nz) * plane;
        const int slot = vs_of<D1>(kk);
        if constexpr (VEC) {
            if (csm < 0) return;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                T* dst = &sm.V[q][slot][csm];
                if (!EVP_STAGE_OK(dst, vel[q] + pv + cvoff[q], E, true)) continue;
                if (cvfac[q] == 1) cp_async16(dst, vel[q] + pv + cvoff[q]);
                else copy_scaled(dst, vel[q] + pv + cvoff[q], cvfac[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int r = 0; r < NV; ++r) {
                    if (psm[r] < 0) continue;
                    T* dst = &sm.V[q][slot][psm[r]];
                    if (!EVP_STAGE_OK(dst, vel[q] + pv + voff[q][r], 1, false)) continue;
                    if (vfac[q][r] == 1)
                        cp_async(dst, vel[q] + pv + voff[q][r]);
                    else
                        *dst = vfac[q][r] == 0 ? T(0) : -__ldg(vel[q] + pv + voff[q][r]);
                }
        }
    };
    auto fetch_p = [&](int kk) {
        const size_t pp = (size_t)wrap1(kk, g.nz) * plane;
        const int slot = ps_of<D1>(kk);
        if constexpr (VEC) {
            if (csm >= 0 && EVP_STAGE_OK(&sm.P[slot][csm], a.P + pp + ccoff, E, true))
                cp_async16(&sm.P[slot][csm], a.P + pp + ccoff);
        } else {
#pragma unroll
            for (int r = 0; r < NV; ++r)
                if (psm[r] >= 0 && EVP_STAGE_OK(&sm.P[slot][psm[r]], a.P + pp + coff[r], 1, false))
                    cp_async(&sm.P[slot][psm[r]], a.P + pp + coff[r]);
        }
    };
    auto fetch_braw = [&](int kk) {
        if constexpr (!SPRE) {
        if (!stress) return;
        const size_t pb = (size_t)wrap1(kk, g.nz) * plane;
        if constexpr (VEC) {
            if (csm < 0) return;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                if (EVP_STAGE_OK(&sm.Braw[kk & 1][c][csm], a.Bo[c] + pb + ccoff, E, true))
                    cp_async16(&sm.Braw[kk & 1][c][csm], a.Bo[c] + pb + ccoff);
                if (EVP_STAGE_OK(&sm.Braw[kk & 1][6 + c][csm], a.Bn[c] + pb + ccoff, E, true))
                    cp_async16(&sm.Braw[kk & 1][6 + c][csm], a.Bn[c] + pb + ccoff);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int r = 0; r < NV; ++r)
                    if (psm[r] >= 0) {
                        if (EVP_STAGE_OK(&sm.Braw[kk & 1][c][psm[r]], a.Bo[c] + pb + coff[r], 1, false))
                            cp_async(&sm.Braw[kk & 1][c][psm[r]], a.Bo[c] + pb + coff[r]);
                        if (EVP_STAGE_OK(&sm.Braw[kk & 1][6 + c][psm[r]], a.Bn[c] + pb + coff[r], 1, false))
                            cp_async(&sm.Braw[kk & 1][6 + c][psm[r]], a.Bn[c] + pb + coff[r]);
                    }
        }
        }
    };
    // shared-memory plane of summed-stress component c at plane kk (kk >= -1): a
    // 3-slot ring built here, a 5-slot ring staged two ahead, or the D1 rings
    auto splane = [&](int c, int kk) -> T* {
        if constexpr (!SPRE) {
            return sm.S[c][pmod(kk, 3)];
        } else if constexpr (!D1) {
            return sm.S[c][vs_of<false>(kk)];
        } else {
            if (c == 2 || c == 4) return sm.S4[c == 2 ? 0 : 1][vs_of<true>(kk)];
            return sm.S3[c < 2 ? c : (c == 3 ? 2 : 3)][ps_of<true>(kk)];
        }
    };
    // precomputed summed stress plane kk into its ring slots (a centred field)
    auto fetch_s = [&](int kk) {
        if constexpr (SPRE) {
            const size_t pb = (size_t)wrap1(kk, g.nz) * plane;
            if constexpr (VEC) {
                if (csm < 0) return;
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (EVP_STAGE_OK(splane(c, kk) + csm, a.S[c] + pb + ccoff, E, true))
                        cp_async16(splane(c, kk) + csm, a.S[c] + pb + ccoff);
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c)
#pragma unroll
                    for (int r = 0; r < NV; ++r)
                        if (psm[r] >= 0 && EVP_STAGE_OK(splane(c, kk) + psm[r], a.S[c] + pb + coff[r], 1, false))
                            cp_async(splane(c, kk) + psm[r], a.S[c] + pb + coff[r]);
            }
        }
    };
    const T kgm = kconst<T>(mc.gmod, mc.f_gmod), kL2 = kconst<T>(mc.L2, mc.f_L2);
    const T kaf = kconst<T>(mc.a_fene, mc.f_a_fene);
    // staged raw B -> summed stress S in ring slot kk mod 3 (Table 1 inverted)
    auto build_s = [&](int kk) {
        if constexpr (!SPRE) {
        if (!stress) return;
        const T gm = kgm;
        const int slot = pmod(kk, 3);
        const T(*Br)[VPL] = sm.Braw[kk & 1];
#pragma unroll
        for (int r = 0; r < NV; ++r) {
            const int e = psm[r];
            if (e < 0) continue;
            if (MODEL == EVP_FENE_P) {
                const T L2 = kL2, av = kaf;
                const T Fo = L2 / (L2 - (Br[0][e] + Br[3][e] + Br[5][e]));
                const T Fn = L2 / (L2 - (Br[6][e] + Br[9][e] + Br[11][e]));
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const bool d = (c == 0 || c == 3 || c == 5);
                    sm.S[c][slot][e] = gm * (Fn * Br[6 + c][e] - (d ? av : T(0)))
                                       + gm * (Fo * Br[c][e] - (d ? av : T(0)));
                }
            } else if (MODEL == EVP_NEO_HOOKEAN) {
                if (a.phis_o) {
                    // soft particles: tau = phi_s G (B - I) at both levels
                    const size_t pb = (size_t)wrap1(kk, g.nz) * plane;
                    const bool pok = EVP_DBG_OK(dbg_src_ok(a.phis_o + pb + coff[r], 1) &&
                                                dbg_src_ok(a.phis_n + pb + coff[r], 1));
                    const T po = pok ? gm * __ldg(a.phis_o + pb + coff[r]) : T(0);
                    const T pn = pok ? gm * __ldg(a.phis_n + pb + coff[r]) : T(0);
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const T d = (c == 0 || c == 3 || c == 5) ? T(1) : T(0);
                        sm.S[c][slot][e] = pn * (Br[6 + c][e] - d) + po * (Br[c][e] - d);
                    }
                } else {
                    // Table 1: tau = G B
#pragma unroll
                    for (int c = 0; c < 6; ++c) sm.S[c][slot][e] = gm * Br[6 + c][e] + gm * Br[c][e];
                }
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const bool d = (c == 0 || c == 3 || c == 5);
                    sm.S[c][slot][e] = gm * (Br[6 + c][e] - (d ? T(1) : T(0)))
                                       + gm * (Br[c][e] - (d ? T(1) : T(0)));
                }
            }
        }
        }
    };
    const size_t cell0 = (size_t)min(j, g.ny - 1) * g.nx + min(i, g.nx - 1);
    // history chunk of this thread (own cells of row hr, columns hq .. hq+E-1)
    constexpr int HCR = TX / E;                          // chunks per tile row
    const int hr = tid / HCR, hq = (tid - hr * HCR) * E;
    const bool hch = VEC && tid < TY * HCR && j0 + hr < g.ny && i0 + hq < g.nx;
    const size_t hoff = (size_t)(j0 + hr) * g.nx + i0 + hq;
    auto fetch_hist = [&](int kk) {
        if (!a.read_hist || kk >= k1) return;
        if constexpr (VEC) {
            if (hch) {
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (EVP_STAGE_OK(&sm.H[hs_of<D1>(kk)][q][hr * TX + hq], a.NH[q] + (size_t)kk * plane + hoff, E, true))
                        cp_async16(&sm.H[hs_of<D1>(kk)][q][hr * TX + hq], a.NH[q] + (size_t)kk * plane + hoff);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (EVP_STAGE_OK(&sm.H[hs_of<D1>(kk)][q][tid], a.NH[q] + (size_t)kk * plane + cell0, 1, false))
                    cp_async(&sm.H[hs_of<D1>(kk)][q][tid], a.NH[q] + (size_t)kk * plane + cell0);
        }
    };

    // ---- prologue: velocity k0-1 .. k0+1, p k0 .. k0+1, S k0-1 .. k0+1, history k0
    // in place; then plane k0+2 and the history of k0+1 requested
    fetch_vel(k0 - 1);
    fetch_vel(k0);
    fetch_vel(k0 + 1);
    fetch_p(k0);
    fetch_p(k0 + 1);
    fetch_hist(k0);
    if constexpr (SPRE) {
        for (int d = -1; d <= 1; ++d) fetch_s(k0 + d);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
    } else {
        for (int d = -1; d <= 1; ++d) {
            fetch_braw(k0 + d);
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
            build_s(k0 + d);
            __syncthreads();
        }
    }
    if constexpr (!D1) {
        fetch_vel(k0 + 2);
        fetch_braw(k0 + 2);
        fetch_s(k0 + 2);
        fetch_p(k0 + 2);
        fetch_hist(k0 + 1);
        cp_async_commit();
    }

    const T h = T(0.5);
    const T idx2 = g.idx * g.idx, idy2 = g.idy * g.idy, idz2 = g.idz * g.idz;
    const T mu = kconst<T>(mc.mu_s, mc.f_mu_s);
    const T two_a = T(2) * a.alpha;
    const int o = (ty + 1) * VW + tx + XO;
    const T* sx_ = a.trig;

    for (int k = k0; k < k1; ++k) {
        // ---- asynchronous request of plane k+3 (velocity, raw B, p) and the history of k+2
        constexpr int AH = D1 ? 2 : 3;
        fetch_vel(k + AH);
        fetch_braw(k + AH);
        fetch_s(k + AH);
        fetch_p(k + AH);
        fetch_hist(k + AH - 1);
        cp_async_commit();

        const int vm1 = vs_of<D1>(k - 1), v0s = vs_of<D1>(k), vp1 = vs_of<D1>(k + 1);
        const T* U0 = sm.V[0][v0s];
        const T* Um1 = sm.V[0][vm1];
        const T* Up1 = sm.V[0][vp1];
        const T* V0 = sm.V[1][v0s];
        const T* Vm1 = sm.V[1][vm1];
        const T* Vp1 = sm.V[1][vp1];
        const T* W0 = sm.V[2][v0s];
        const T* Wm1 = sm.V[2][vm1];
        const T* Wp1 = sm.V[2][vp1];
        // value at (i+di, j+dj) of a plane
        auto at = [&](const T* Pl, int di, int dj) { return Pl[o + dj * VW + di]; };
        const T u0 = at(U0, 0, 0), v0 = at(V0, 0, 0), w0 = at(W0, 0, 0);

        // ---- div(uu) at the three faces
        const T Ax = (sq(h * (u0 + at(U0, 1, 0))) - sq(h * (at(U0, -1, 0) + u0))) * g.idx
                     + (h * (u0 + at(U0, 0, 1)) * h * (v0 + at(V0, 1, 0))
                        - h * (at(U0, 0, -1) + u0) * h * (at(V0, 0, -1) + at(V0, 1, -1))) * g.idy
                     + (h * (u0 + at(Up1, 0, 0)) * h * (w0 + at(W0, 1, 0))
                        - h * (at(Um1, 0, 0) + u0) * h * (at(Wm1, 0, 0) + at(Wm1, 1, 0))) * g.idz;
        const T Ay = (h * (u0 + at(U0, 0, 1)) * h * (v0 + at(V0, 1, 0))
                      - h * (at(U0, -1, 0) + at(U0, -1, 1)) * h * (at(V0, -1, 0) + v0)) * g.idx
                     + (sq(h * (v0 + at(V0, 0, 1))) - sq(h * (at(V0, 0, -1) + v0))) * g.idy
                     + (h * (v0 + at(Vp1, 0, 0)) * h * (w0 + at(W0, 0, 1))
                        - h * (at(Vm1, 0, 0) + v0) * h * (at(Wm1, 0, 0) + at(Wm1, 0, 1))) * g.idz;
        const T Az = (h * (u0 + at(Up1, 0, 0)) * h * (w0 + at(W0, 1, 0))
                      - h * (at(U0, -1, 0) + at(Up1, -1, 0)) * h * (at(W0, -1, 0) + w0)) * g.idx
                     + (h * (v0 + at(Vp1, 0, 0)) * h * (w0 + at(W0, 0, 1))
                        - h * (at(V0, 0, -1) + at(Vp1, 0, -1)) * h * (at(W0, 0, -1) + w0)) * g.idy
                     + (sq(h * (w0 + at(Wp1, 0, 0))) - sq(h * (at(Wm1, 0, 0) + w0))) * g.idz;

        // ---- mu_s lap(u)
        const T Lu = (at(U0, 1, 0) - T(2) * u0 + at(U0, -1, 0)) * idx2 + (at(U0, 0, 1) - T(2) * u0 + at(U0, 0, -1)) * idy2
                     + (at(Up1, 0, 0) - T(2) * u0 + at(Um1, 0, 0)) * idz2;
        const T Lv = (at(V0, 1, 0) - T(2) * v0 + at(V0, -1, 0)) * idx2 + (at(V0, 0, 1) - T(2) * v0 + at(V0, 0, -1)) * idy2
                     + (at(Vp1, 0, 0) - T(2) * v0 + at(Vm1, 0, 0)) * idz2;
        const T Lw = (at(W0, 1, 0) - T(2) * w0 + at(W0, -1, 0)) * idx2 + (at(W0, 0, 1) - T(2) * w0 + at(W0, 0, -1)) * idy2
                     + (at(Wp1, 0, 0) - T(2) * w0 + at(Wm1, 0, 0)) * idz2;

        // ---- body force: uniform dp/dx plus ABC forcing (separable tables)
        T fx = a.dpdx, fy = T(0), fz = T(0);
        if (sx_ && active) {
            const T* cx = sx_ + g.nx;
            const T* sy = cx + g.nx;
            const T* cy = sy + g.ny;
            const T* sz = cy + g.ny;
            const T* cz = sz + g.nz;
            fx += a.abc_amp * (__ldg(sz + k) + __ldg(cy + j));
            fy = a.abc_amp * (__ldg(sx_ + i) + __ldg(cz + k));
            fz = a.abc_amp * (__ldg(sy + j) + __ldg(cx + i));
        }
        // implicit viscous option: the viscous term leaves N (alpha mu lap u^{k-1} is
        // added below; alpha mu lap u* is taken by the Helmholtz solves)
        const T mun = a.cn ? T(0) : mu;
        const T Nx = -Ax + mun * Lu + fx;
        const T Ny = -Ay + mun * Lv + fy;
        const T Nz = -Az + mun * Lw + fz;

        // ---- pressure gradient
        const T* P0 = sm.P[ps_of<D1>(k)];
        const T* P1 = sm.P[ps_of<D1>(k + 1)];
        const T p0 = at(P0, 0, 0);
        const T gpx = (at(P0, 1, 0) - p0) * g.idx;
        const T gpy = (at(P0, 0, 1) - p0) * g.idy;
        const T gpz = (at(P1, 0, 0) - p0) * g.idz;

        T ix = a.zeta * Nx, iy = a.zeta * Ny, iz = a.zeta * Nz;
        if (a.read_hist) {
            ix += a.xi * sm.H[hs_of<D1>(k)][0][tid];
            iy += a.xi * sm.H[hs_of<D1>(k)][1][tid];
            iz += a.xi * sm.H[hs_of<D1>(k)][2][tid];
        }
        ix -= two_a * gpx;
        iy -= two_a * gpy;
        iz -= two_a * gpz;
        if (a.cn) {
            const T am = a.alpha * mu;
            ix += am * Lu;
            iy += am * Lv;
            iz += am * Lw;
        }
        if (stress) {
            // planes k, k-1 and k+1 (the ring slot of each component comes from splane)
            const int s0 = k, sm1 = k - 1, sp1 = k + 1;
            auto S = [&](int c, int kk, int di, int dj) { return splane(c, kk)[o + dj * VW + di]; };
            // 4-point average over centres (0 or di) x (0 or dj) in one plane
            auto e4 = [&](int c, int slot, int di, int dj) {
                return T(0.25) * (S(c, slot, 0, 0) + S(c, slot, 0, dj) + S(c, slot, di, 0) + S(c, slot, di, dj));
            };
            // 4-point average over (0 or di) x planes (k, k+dk) at row j, or (0 or dj) x planes
            auto e4z = [&](int c, int di, int dj, int slot2) {
                return T(0.25) * (S(c, s0, 0, 0) + S(c, slot2, 0, 0) + S(c, s0, di, dj) + S(c, slot2, di, dj));
            };
            const T fxs = (S(0, s0, 1, 0) - S(0, s0, 0, 0)) * g.idx
                          + (e4(1, s0, 1, 1) - e4(1, s0, 1, -1)) * g.idy
                          + (e4z(2, 1, 0, sp1) - e4z(2, 1, 0, sm1)) * g.idz;
            const T fys = (e4(1, s0, 1, 1) - e4(1, s0, -1, 1)) * g.idx
                          + (S(3, s0, 0, 1) - S(3, s0, 0, 0)) * g.idy
                          + (e4z(4, 0, 1, sp1) - e4z(4, 0, 1, sm1)) * g.idz;
            const T fzs = (e4z(2, 1, 0, sp1) - e4z(2, -1, 0, sp1)) * g.idx
                          + (e4z(4, 0, 1, sp1) - e4z(4, 0, -1, sp1)) * g.idy
                          + (S(5, sp1, 0, 0) - S(5, s0, 0, 0)) * g.idz;
            ix += a.alpha * fxs;
            iy += a.alpha * fys;
            iz += a.alpha * fzs;
        }
        if (active && EVP_DBG_OK((size_t)k * plane + (size_t)j * g.nx + i < plane * (size_t)g.nz)) {
            const size_t c0 = (size_t)k * plane + (size_t)j * g.nx + i;
            T us = u0 + a.dt * ix, vs = v0 + a.dt * iy, ws = w0 + a.dt * iz;
            if (a.solid[0]) {
                // volume penalisation of fixed obstacles, Eq. forceAdded
                us *= T(1) - __ldg(a.solid[0] + c0);
                vs *= T(1) - __ldg(a.solid[1] + c0);
                ws *= T(1) - __ldg(a.solid[2] + c0);
            }
            a.Us[c0] = us;
            a.Vs[c0] = (g.walls && j == g.ny - 1) ? T(0) : vs;
            a.Ws[c0] = ws;
            if (a.write_hist) {
                a.NH[0][c0] = Nx;
                a.NH[1][c0] = Ny;
                a.NH[2][c0] = Nz;
            }
        }

        // ---- advance: plane k+2 has landed (only plane k+3 may be in flight); its
        // raw B becomes S plane k+2 (slot of plane k-1).  With the precomputed
        // stress every ring slot written at the next plane was last read before
        // this barrier, which is the only one per plane.
        if constexpr (D1) cp_async_wait_all();   // plane k+2 has landed
        else cp_async_wait_prev();
        __syncthreads();
        if constexpr (!SPRE) {
            build_s(k + 2);
            __syncthreads();
        }
    }
    // two-plane staging: the last request (two planes past the chunk) may still be
    // in flight; let it land before the tile's shared memory is given up
    if constexpr (!D1) cp_async_wait_all();
    EVP_DBG_REPORT(a.status);
}

template <typename T, int MODEL, bool VEC, bool SPRE>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 2)
k_momentum(const Geo<T> g, const ModelConst mc, const MomentumArgs<T> a, int kz_chunk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    momentum_tile<T, MODEL, VEC, SPRE>(g, mc, a, kz_chunk, blockIdx.x, blockIdx.y, blockIdx.z, smraw);
}

// the precomputed-stress kernel staged one plane ahead, six CTAs per SM in FP32
template <typename T, bool VEC>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 6 : 2)
k_momentum_d1(const Geo<T> g, const ModelConst mc, const MomentumArgs<T> a, int kz_chunk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    momentum_tile<T, EVP_OLDROYD_B, VEC, true, true>(g, mc, a, kz_chunk, blockIdx.x, blockIdx.y, blockIdx.z, smraw);
}

// Batched form (summed stress precomputed): a persistent grid walks a work list
// of (member, tile x, tile y, z chunk); members' grids may differ.
template <typename T, bool VEC>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 2)
k_momentum_batch(const __grid_constant__ MomentumBatch<T> p, const int4* __restrict__ work, int nwork) {
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int4 t = __ldg(work + w);
        const MomentumMember<T>& m = p.m[t.x];
        momentum_tile<T, EVP_OLDROYD_B, VEC, true>(m.g, m.mc, m.a, m.kz, t.y, t.z, t.w, smraw);
        __syncthreads();
    }
}

}  // namespace

template <typename T>
cudaError_t launch_momentum(const Geo<T>& g, const ModelConst& mc, const MomentumArgs<T>& a,
                            cudaStream_t st, const TimingHook& th) {
    // z chunks: about four waves of CTAs; small grids go down to one plane per CTA
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    const int per_sm = sizeof(T) == 4 ? 4 : 2;
    int chunks = (4 * 152 * per_sm + tiles - 1) / tiles;
    chunks = chunks > g.nz ? g.nz : chunks;
    const int kz = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + kz - 1) / kz;
    dim3 block(TX, TY, 1);
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, chunks);
    const bool vec = (g.nx * sizeof(T)) % 16 == 0;
    if (a.S[0] && sizeof(T) == 4) {
        // summed stress precomputed by the stress kernel: staged one plane ahead
        if (mc.model == EVP_NEWTONIAN) return cudaErrorInvalidValue;
        const size_t smem = sizeof(MomSmemS1<T>);
        int ch = (4 * 152 * 6 + tiles - 1) / tiles;
        ch = ch > g.nz ? g.nz : ch;
        const int kz1 = (g.nz + ch - 1) / ch;
        ch = (g.nz + kz1 - 1) / kz1;
        const dim3 grid1((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, ch);
        th.b(K_MOMENTUM);
        auto kern = vec ? k_momentum_d1<T, true> : k_momentum_d1<T, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // all of the SM's unified L1 / shared memory as shared memory: six CTAs of 36.7 KB
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (cudaError_t e = launch_k(kern, grid1, block, smem, st, th.pdl, g, mc, a, kz1)) return e;
        th.e(K_MOMENTUM);
        return cudaGetLastError();
    }
    if (a.S[0]) {
        // summed stress precomputed by the stress kernel
        if (mc.model == EVP_NEWTONIAN) return cudaErrorInvalidValue;
        const size_t smem = sizeof(MomSmemS<T>);
        th.b(K_MOMENTUM);
        auto kern = vec ? k_momentum<T, EVP_OLDROYD_B, true, true> : k_momentum<T, EVP_OLDROYD_B, false, true>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (cudaError_t e = launch_k(kern, grid, block, smem, st, th.pdl, g, mc, a, kz)) return e;
        th.e(K_MOMENTUM);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(MomSmem<T>);
    th.b(K_MOMENTUM);
    switch (mc.model * 2 + (vec ? 1 : 0)) {
#define EVP_LAUNCH_MOM_V(M, V)                                                                                       \
    case M * 2 + V:                                                                                                  \
        cudaFuncSetAttribute(k_momentum<T, M, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        if (cudaError_t e = launch_k(k_momentum<T, M, V, false>, grid, block, smem, st, th.pdl, g, mc, a, kz))     \
            return e;                                                                                                 \
        break;
#define EVP_LAUNCH_MOM(M) EVP_LAUNCH_MOM_V(M, false) EVP_LAUNCH_MOM_V(M, true)
        EVP_LAUNCH_MOM(EVP_NEWTONIAN)
        EVP_LAUNCH_MOM(EVP_OLDROYD_B)
        EVP_LAUNCH_MOM(EVP_FENE_P)
        EVP_LAUNCH_MOM(EVP_SARAMITO)
        EVP_LAUNCH_MOM(EVP_NEO_HOOKEAN)
#undef EVP_LAUNCH_MOM
#undef EVP_LAUNCH_MOM_V
        default: return cudaErrorInvalidValue;
    }
    th.e(K_MOMENTUM);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_momentum_batch(const MomentumBatch<T>& p, bool vec, const int4* work, int nwork, int ctas,
                                  cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    const size_t smem = sizeof(MomSmemS<T>);
    const dim3 grid(ctas < nwork ? ctas : nwork), block(TX, TY, 1);
    auto kern = vec ? k_momentum_batch<T, true> : k_momentum_batch<T, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_k(kern, grid, block, smem, st, false, p, work, nwork);
}

int momentum_tile_x() { return TX; }
int momentum_tile_y() { return TY; }
template <typename T>
int momentum_ctas_per_sm() { return sizeof(T) == 4 ? 4 : 2; }

template cudaError_t launch_momentum_batch<float>(const MomentumBatch<float>&, bool, const int4*, int, int,
                                                  cudaStream_t);
template cudaError_t launch_momentum_batch<double>(const MomentumBatch<double>&, bool, const int4*, int, int,
                                                   cudaStream_t);
template int momentum_ctas_per_sm<float>();
template int momentum_ctas_per_sm<double>();

template cudaError_t launch_momentum<float>(const Geo<float>&, const ModelConst&, const MomentumArgs<float>&,
                                            cudaStream_t, const TimingHook&);
template cudaError_t launch_momentum<double>(const Geo<double>&, const ModelConst&, const MomentumArgs<double>&,
                                             cudaStream_t, const TimingHook&);

}  // namespace evp
