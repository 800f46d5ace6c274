// S1 + S2: centre velocity and velocity gradient, WENO5 advection of the six
// components of B, the Table 1 closure and the RK3 update of Eq. rk3tau.
//
// RT = (a I - F B)/lambda - (u.grad B - B.grad u - grad u^T.B)     (Eq. rt / RK-rt)
//      [+ kappa_ad lap B where det B < 0 or, FENE-P, tr B >= 0.95 L^2  (Sec. 3.1)]
// B^k = B^{k-1} + dt (zeta^k RT^{k-1} + xi^k RT^{k-2})            (Eq. rk3tau)
//
// z-marching tiles: see the kernel for the data staging.  The kernel template is
// instantiated once per precision, in k_stress_f32.cu and k_stress_f64.cu.
#pragma once
#include <cfloat>

#include "evp_internal.cuh"
#include "weno.cuh"

namespace evp {

namespace {

// storage index of the symmetric component (a, b): xx xy xz yy yz zz
__device__ __forceinline__ constexpr int symi(int a, int b) {
    return a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5));
}
__device__ __forceinline__ constexpr int row_of(int c) { return c < 3 ? 0 : (c < 5 ? 1 : 2); }
__device__ __forceinline__ constexpr int col_of(int c) { return c == 0 ? 0 : ((c == 1 || c == 3) ? 1 : 2); }


// Tile geometry of the z-marching kernel: a 32 x 8 tile of cells in x-y walks
// through a chunk of z planes.  B of the tile's own columns lives in an 8-plane
// shared-memory ring (planes k-3 .. k+3 for the z stencils, k+4 arriving); the
// current plane of B with a 3-cell x-y halo and three planes of u, v, w with a
// 1-cell halo live in shared memory too.  Plane
// rows are 40 wide with the tile's i0 at column 4 (x = i0-4 .. i0+35), so that
// when nx is a whole number of 16-byte chunks every row is staged in 16-byte
// cp.async chunks; other grids stage element by element.
constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int XO = 4;                                     // column of x = i0 in a plane row
constexpr int BW = TX + 8, BH = TY + 6, BPL = BW * BH;    // B plane rows j0-3 .. j0+10
constexpr int VW = TX + 8, VH = TY + 2, VPL = VW * VH;    // velocity plane rows j0-1 .. j0+8
constexpr int BHALO = (TX + 6) * BH - NT;                 // 276 halo cells the stencils use
constexpr int NBH = (BHALO + NT - 1) / NT;                // halo cells per thread (2)
constexpr int VUSED = (TX + 2) * VH;                      // velocity cells the stencils use
constexpr int NVH = (VUSED + NT - 1) / NT;                // velocity cells per thread (2)

__device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}
// a in [-n, 2n): one conditional wrap, no division
__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// (row, x - (i0-3)) of used halo cell h (0 <= h < 276) of a B plane: three full
// rows above and below the tile, three cells left and right of its 8 rows
__device__ __forceinline__ void bhalo_pos(int h, int& hy, int& hx) {
    constexpr int W = TX + 6;
    if (h < 3 * W) {
        hy = h / W;
        hx = h % W;
    } else if (h < 6 * W) {
        const int q = h - 3 * W;
        hy = TY + 3 + q / W;
        hx = q % W;
    } else {
        const int q = h - 6 * W;
        hy = 3 + q / 6;
        const int c = q % 6;
        hx = c < 3 ? c : TX + c;
    }
}

// chunk h (16 bytes, E elements) of the halo ring of a B plane: whole rows 0..2
// and BH-3..BH-1, and the chunks covering columns 0..3 and TX+4..TX+7 of rows
// 3..BH-4.  Returns (row, first column).
template <int E>
__device__ __forceinline__ void bring_pos(int h, int& row, int& col) {
    constexpr int CPR = BW / E, LC = XO / E;
    if (h < 6 * CPR) {
        const int r = h / CPR;
        row = r < 3 ? r : BH - 6 + r;
        col = (h - r * CPR) * E;
    } else {
        const int q = h - 6 * CPR;
        const int r = q / (2 * LC), s = q - r * (2 * LC);
        row = 3 + r;
        col = s < LC ? s * E : TX + XO + (s - LC) * E;
    }
}

// 16-byte asynchronous copy (L2 only)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <typename T>
struct StressSmem {
    T B[2][6][BPL];     // plane k (being used) and plane k+1 (arriving) of B, 3-cell halo
    T V[3][4][VPL];     // [u, v, w][ring slot: planes k-1 .. k+2][plane with 1-cell halo]
    T N[8][6][NT];      // ring of B planes k-3 .. k+4 for the tile's own columns (slot = plane & 7)
    T H[2][6][NT];      // RK3 history RT^{k-2} of planes k and k+1 for the tile's cells
};

// asynchronous global -> shared copy of one element (cp.async, L1-allocating)
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

// MODE: 0 = right-hand side only, 1 = update without history read (first RK3
// substep / first AB2 step), 2 = update reading and writing the history,
// 3 = update reading the history without writing it (last RK3 substep).
// DIFF: the local artificial diffusion is on (ModelConst::art_diff > 0).
// VEC: planes are staged in 16-byte chunks (needs nx * sizeof(T) % 16 == 0).
// One tile: the 32 x 8 columns (bx, by) over the z chunk bz of kz_chunk planes.
template <typename T, int MODEL, int MODE, bool DIFF, bool VEC>
__device__ __forceinline__ void stress_tile(const Geo<T>& g, const ModelConst& mc, const StressArgs<T>& a,
                                            int kz_chunk, int bx, int by, int bz, unsigned char* smraw) {
    constexpr bool RHS_ONLY = MODE == 0, READ_H = MODE >= 2, WRITE_H = MODE == 1 || MODE == 2;
    StressSmem<T>& sm = *reinterpret_cast<StressSmem<T>*>(smraw);
    EVP_DBG_DECL;
#ifdef EVP_DEBUG
    dbg_poison(smraw, sizeof(StressSmem<T>));
    const size_t dbg_n = (size_t)g.nx * g.ny * g.nz;
    auto dbg_src_ok = [&](const T* p, int n) {
        if (dbg_within(p, n, a.U, dbg_n) || dbg_within(p, n, a.V, dbg_n) || dbg_within(p, n, a.W, dbg_n) ||
            dbg_within(p, n, a.H, dbg_n))
            return true;
        for (int c = 0; c < 6; ++c)
            if (dbg_within(p, n, a.B[c], dbg_n) || dbg_within(p, n, (const T*)a.RT[c], dbg_n)) return true;
        return false;
    };
    auto dbg_dst_ok = [&](const T* d, int n) {
        return (const unsigned char*)d >= smraw && (const unsigned char*)(d + n) <= smraw + sizeof(StressSmem<T>);
    };
#endif
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = bx * TX, j0 = by * TY;
    const int k0 = bz * kz_chunk;
    const int k1 = min(k0 + kz_chunk, g.nz);
    const int i = i0 + tx, j = j0 + ty;
    const bool active = (i < g.nx) && (j < g.ny);
    const size_t plane = (size_t)g.nx * g.ny;
    // the column this thread loads (wrapped / clamped so that ragged threads hold
    // the periodic or ghost image their neighbours' stencils need)
    const int jc = g.walls ? min(j, g.ny - 1) : pmod(j, g.ny);
    const size_t col = (size_t)jc * g.nx + pmod(i, g.nx);

    // ---- row ghost rules (walls): centred fields copy the nearest row, u and w
    // take the odd mirror (no slip), v is zero outside the stored faces; a
    // periodic y wraps.  Returns the source row and the factor (+1 copy, -1
    // negated copy, 0 zero) of velocity component q, or of B for q = 3.
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
    constexpr int E = 16 / (int)sizeof(T);             // elements per 16-byte chunk
    constexpr int CPR = BW / E;                        // chunks per plane row
    constexpr int RING = 6 * CPR + 2 * TY * (XO / E);  // halo-ring chunks of a B plane
    constexpr int NRC = (6 * RING + NT - 1) / NT;      // ring copies per thread (6 fields)
    constexpr int VCH = CPR * VH;                      // chunks of a velocity plane
    constexpr int OCH = TY * (TX / E);                 // chunks of the tile's own cells
    constexpr int NOC = (6 * OCH + NT - 1) / NT;       // own-cell copies per thread (6 fields)

    // element-wise staging (VEC false): this thread's B halo and velocity cells
    size_t hoff[NBH];
    int hsm[NBH];
    size_t voff[3][NVH];
    signed char vfac[3][NVH];
    int vsm[NVH];
    // chunk staging (VEC true): the source of each copy in plane 0 (a plane's copy
    // adds its plane offset) and its shared-memory offset, for the ring copies, the
    // velocity chunk and the own-cell chunks of B and of the history
    const T* rc_src[NRC];
    int rc_sm[NRC];
    int csm = -1;
    const T* cv_src[3] = {a.U, a.V, a.W};
    signed char cvfac[3] = {0, 0, 0};
    const T* oc_src[NOC];
    const T* oc_hsrc[NOC];
    int oc_sm[NOC];
    bool oc_act[NOC];
    if (VEC) {
#pragma unroll
        for (int r = 0; r < NRC; ++r) {
            const int idx = tid + r * NT;
            rc_sm[r] = -1;
            rc_src[r] = a.B[0];
            if (idx < 6 * RING) {
                const int c = idx / RING, h = idx - c * RING;
                int row, colq;
                bring_pos<E>(h, row, colq);
                int src;
                row_rule(j0 + row - 3, 3, src);
                rc_src[r] = a.B[c] + (size_t)src * g.nx + pmod(i0 - XO + colq, g.nx);
                rc_sm[r] = c * BPL + row * BW + colq;
            }
        }
        if (tid < VCH) {
            const int r = tid / CPR, q0 = (tid - r * CPR) * E;
            csm = r * VW + q0;
            const int gx = pmod(i0 - XO + q0, g.nx);
            int src;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                cvfac[q] = (signed char)row_rule(j0 - 1 + r, q, src);
                cv_src[q] += (size_t)src * g.nx + gx;
            }
        }
#pragma unroll
        for (int r = 0; r < NOC; ++r) {
            const int idx = tid + r * NT;
            oc_sm[r] = -1;
            oc_src[r] = a.B[0];
            oc_hsrc[r] = a.RT[0];
            oc_act[r] = false;
            if (idx < 6 * OCH) {
                const int c = idx / OCH, h = idx - c * OCH;
                const int row = h / (TX / E), q0 = (h - row * (TX / E)) * E;
                int src;
                row_rule(j0 + row, 3, src);
                oc_src[r] = a.B[c] + (size_t)src * g.nx + pmod(i0 + q0, g.nx);
                oc_sm[r] = c * NT + row * TX + q0;
                oc_act[r] = j0 + row < g.ny && i0 + q0 < g.nx;
                oc_hsrc[r] = a.RT[c] + (size_t)(j0 + row) * g.nx + i0 + q0;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NBH; ++r) {
        const int h = tid + r * NT;
        hsm[r] = -1;
        hoff[r] = 0;
        if (!VEC && h < BHALO) {
            int hy, hx;
            bhalo_pos(h, hy, hx);
            int src;
            row_rule(j0 + hy - 3, 3, src);
            hoff[r] = (size_t)src * g.nx + pmod(i0 + hx - 3, g.nx);
            hsm[r] = hy * BW + hx + XO - 3;
        }
    }
#pragma unroll
    for (int r = 0; r < NVH; ++r) {
        const int e = tid + r * NT;
        const int vy = e / (TX + 2), vx = e - vy * (TX + 2);
        vsm[r] = (!VEC && e < VUSED) ? vy * VW + vx + XO - 1 : -1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            voff[q][r] = 0;
            vfac[q][r] = 0;
        }
        if (vsm[r] < 0) continue;
        const int gx = pmod(i0 + vx - 1, g.nx);
        int src;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            vfac[q][r] = (signed char)row_rule(j0 + vy - 1, q, src);
            voff[q][r] = (size_t)src * g.nx + gx;
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
    // velocity plane kk (unwrapped index) into ring slot kk mod 4
    auto fetch_vel = [&](int kk) {
        const size_t pv = (size_t)wrap1(kk, g.nz) * plane;
        const int slot = kk & 3;
        if constexpr (VEC) {
            if (csm < 0) return;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                T* dst = &sm.V[q][slot][csm];
                if (!EVP_STAGE_OK(dst, cv_src[q] + pv, E, true)) continue;
                if (cvfac[q] == 1) cp_async16(dst, cv_src[q] + pv);
                else copy_scaled(dst, cv_src[q] + pv, cvfac[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int r = 0; r < NVH; ++r) {
                    if (vsm[r] < 0) continue;
                    T* dst = &sm.V[q][slot][vsm[r]];
                    if (!EVP_STAGE_OK(dst, vel[q] + pv + voff[q][r], 1, false)) continue;
                    if (vfac[q][r] == 1)
                        cp_async(dst, vel[q] + pv + voff[q][r]);
                    else
                        *dst = vfac[q][r] == 0 ? T(0) : -__ldg(vel[q] + pv + voff[q][r]);
                }
        }
    };
    // halo ring of B plane kk into buffer kk & 1
    auto fetch_halo = [&](int kk) {
        const size_t ph = (size_t)wrap1(kk, g.nz) * plane;
        const int buf = kk & 1;
        if constexpr (VEC) {
#pragma unroll
            for (int r = 0; r < NRC; ++r)
                if (rc_sm[r] >= 0 && EVP_STAGE_OK(&sm.B[buf][0][0] + rc_sm[r], rc_src[r] + ph, E, true))
                    cp_async16(&sm.B[buf][0][0] + rc_sm[r], rc_src[r] + ph);
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c)
#pragma unroll
                for (int r = 0; r < NBH; ++r)
                    if (hsm[r] >= 0 && EVP_STAGE_OK(&sm.B[buf][c][hsm[r]], a.B[c] + ph + hoff[r], 1, false))
                        cp_async(&sm.B[buf][c][hsm[r]], a.B[c] + ph + hoff[r]);
        }
    };
    // plane kk of B for the tile's own columns into ring slot kk & 7 (kk >= -nz)
    auto fetch_next = [&](int kk) {
        const size_t pb = (size_t)wrap1(kk, g.nz) * plane;
        T* slot = &sm.N[kk & 7][0][0];
        if constexpr (VEC) {
#pragma unroll
            for (int r = 0; r < NOC; ++r)
                if (oc_sm[r] >= 0 && EVP_STAGE_OK(slot + oc_sm[r], oc_src[r] + pb, E, true))
                    cp_async16(slot + oc_sm[r], oc_src[r] + pb);
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c)
                if (EVP_STAGE_OK(slot + c * NT + tid, a.B[c] + pb + col, 1, false))
                    cp_async(slot + c * NT + tid, a.B[c] + pb + col);
        }
    };

    // ---- prologue: the own-column ring (planes k0-3 .. k0+3), velocity planes
    // k0-1 .. k0+1, the halo of plane k0; then its interior from the ring
#pragma unroll 1
    for (int m = -3; m <= 3; ++m) fetch_next(k0 + m);
    fetch_vel(k0 - 1);
    fetch_vel(k0);
    fetch_vel(k0 + 1);
    fetch_halo(k0);
    // RK3 history of this thread's cell in plane kk -> staging buffer kk & 1
    const size_t cell0 = (size_t)j * g.nx + i;
    auto fetch_hist = [&](int kk) {
        if constexpr (READ_H) {
            if (kk >= k1) return;
            if constexpr (VEC) {
#pragma unroll
                for (int r = 0; r < NOC; ++r)
                    if (oc_sm[r] >= 0 && oc_act[r] &&
                        EVP_STAGE_OK(&sm.H[kk & 1][0][0] + oc_sm[r], oc_hsrc[r] + (size_t)kk * plane, E, true))
                        cp_async16(&sm.H[kk & 1][0][0] + oc_sm[r], oc_hsrc[r] + (size_t)kk * plane);
            } else {
                if (!active) return;
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    if (EVP_STAGE_OK(&sm.H[kk & 1][c][tid], a.RT[c] + (size_t)kk * plane + cell0, 1, false))
                        cp_async(&sm.H[kk & 1][c][tid], a.RT[c] + (size_t)kk * plane + cell0);
            }
        }
    };
    fetch_hist(k0);
    const int ob = (ty + 3) * BW + tx + XO;   // this cell in a B plane
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 6; ++c) sm.B[k0 & 1][c][ob] = sm.N[k0 & 7][c][tid];
    __syncthreads();

    const T inv_lam = kconst<T>(mc.inv_lam, mc.f_inv_lam);
    const T kL2 = kconst<T>(mc.L2, mc.f_L2), kaf = kconst<T>(mc.a_fene, mc.f_a_fene);
    const T kgm = kconst<T>(mc.gmod, mc.f_gmod), kty = kconst<T>(mc.tau_y, mc.f_tau_y);
    const T dtz = a.dt_zeta, dtx = a.dt_xi;
    const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
    const int o = (ty + 1) * VW + tx + XO;    // this cell in a velocity plane
    unsigned bits = 0;

    for (int k = k0; k < k1; ++k) {
        // ---- plane k+1 of B: the interior from the ring, the halo by asynchronous
        // copy; asynchronous prefetch of plane k+4 (own columns), velocity plane k+2
        // and history plane k+1.  Every buffer written here was last read before
        // the previous plane's barrier, the only one per plane.
        {
#pragma unroll
            for (int c = 0; c < 6; ++c) sm.B[(k + 1) & 1][c][ob] = sm.N[(k + 1) & 7][c][tid];
            fetch_next(k + 4);
            fetch_halo(k + 1);
            fetch_vel(k + 2);
            fetch_hist(k + 1);
            cp_async_commit();
        }

        // ---- S1: centre velocity and gradient (Reading 5) from the velocity ring
        const T* Up_ = sm.V[0][((k - 1) & 3)];
        const T* Uc_ = sm.V[0][(k & 3)];
        const T* Un_ = sm.V[0][((k + 1) & 3)];
        const T* Vp_ = sm.V[1][((k - 1) & 3)];
        const T* Vc_ = sm.V[1][(k & 3)];
        const T* Vn_ = sm.V[1][((k + 1) & 3)];
        const T* Wp_ = sm.V[2][((k - 1) & 3)];
        const T* Wc_ = sm.V[2][(k & 3)];
        const T Uc = Uc_[o], Um = Uc_[o - 1];
        const T Vc = Vc_[o], Vm = Vc_[o - VW];
        const T Wc = Wc_[o], Wm = Wp_[o];
        const T uc = T(0.5) * (Um + Uc), vc = T(0.5) * (Vm + Vc), wc = T(0.5) * (Wm + Wc);
        T L[3][3];
        L[0][0] = (Uc - Um) * g.idx;
        L[1][1] = (Vc - Vm) * g.idy;
        L[2][2] = (Wc - Wm) * g.idz;
        L[0][1] = (T(0.5) * (Uc_[o + VW - 1] + Uc_[o + VW]) - T(0.5) * (Uc_[o - VW - 1] + Uc_[o - VW])) * hy;
        L[0][2] = (T(0.5) * (Un_[o - 1] + Un_[o]) - T(0.5) * (Up_[o - 1] + Up_[o])) * hz;
        L[1][0] = (T(0.5) * (Vc_[o + 1 - VW] + Vc_[o + 1]) - T(0.5) * (Vc_[o - 1 - VW] + Vc_[o - 1])) * hx;
        L[1][2] = (T(0.5) * (Vn_[o - VW] + Vn_[o]) - T(0.5) * (Vp_[o - VW] + Vp_[o])) * hz;
        L[2][0] = (T(0.5) * (Wp_[o + 1] + Wc_[o + 1]) - T(0.5) * (Wp_[o - 1] + Wc_[o - 1])) * hx;
        L[2][1] = (T(0.5) * (Wp_[o + VW] + Wc_[o + VW]) - T(0.5) * (Wp_[o - VW] + Wc_[o - VW])) * hy;

        // ---- B^{k-1} of the cell (ring slot of plane k)
        const T* Nf = &sm.N[0][0][0];
        T b0[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) b0[c] = sm.N[k & 7][c][tid];

        // ---- Table 1 closure at the cell
        T F = T(1), av = T(1);
        if (MODEL == EVP_NEO_HOOKEAN) {
            F = T(0);
            av = T(0);
        } else if (MODEL == EVP_FENE_P) {
            const T tr = b0[0] + b0[3] + b0[5];
            if (sizeof(T) == 4) F = kL2 * T(rcp_approx(float(kL2 - tr)));
            else F = kL2 / (kL2 - tr);
            av = kaf;
        } else if (MODEL == EVP_SARAMITO) {
            T gm = kgm;
            if (a.H) {
                // two-phase mixture: polymer viscosity mu_p(H) of the cell
                const T* hp = a.H + (size_t)k * plane + col;
                const T Hc = EVP_DBG_OK(dbg_src_ok(hp, 1)) ? __ldg(hp) : T(0);
                gm = (a.mu_p1 * Hc + a.mu_p2 * (T(1) - Hc)) * inv_lam;
            }
            T t[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) t[c] = gm * (b0[c] - ((c == 0 || c == 3 || c == 5) ? T(1) : T(0)));
            const T tr3 = (t[0] + t[3] + t[5]) * T(1.0 / 3.0);
            const T d0 = t[0] - tr3, d3 = t[3] - tr3, d5 = t[5] - tr3;
            const T mag2 = T(0.5) * (d0 * d0 + d3 * d3 + d5 * d5) + t[1] * t[1] + t[2] * t[2] + t[4] * t[4];
            const T tyv = kty;
            if (sizeof(T) == 4) {
                // F = max(0, 1 - tau_y/|tau^d|) with the approximate reciprocal square
                // root instruction; tau_y = 0 is exactly Oldroyd-B (F = 1)
                float rs;
                asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(float(mag2)));
                const T f = T(1) - tyv * T(rs);
                F = tyv > T(0) ? (mag2 > T(0) && f > T(0) ? f : T(0)) : T(1);
            } else if (mag2 > T(0)) {
                const T f = T(1) - tyv / sqrt(mag2);
                F = f > T(0) ? f : T(0);
            } else {
                F = tyv > T(0) ? T(0) : T(1);
            }
            av = F;
        }

        // ---- local artificial diffusion (Sec. 3.1): selected from B^{k-1} of the cell
        T kad = T(0);
        if constexpr (DIFF) {
            const T det0 = b0[0] * (b0[3] * b0[5] - b0[4] * b0[4]) - b0[1] * (b0[1] * b0[5] - b0[4] * b0[2])
                           + b0[2] * (b0[1] * b0[4] - b0[3] * b0[2]);
            bool hit = det0 < T(0);
            if (MODEL == EVP_FENE_P) hit = hit || (b0[0] + b0[3] + b0[5] >= T(0.95) * kL2);
            kad = hit ? kconst<T>(mc.art_diff, mc.f_art_diff) : T(0);
        }

        // ---- WENO5 advection (stencil direction +1 for a positive velocity), UCD, update
        const int sx = uc > T(0) ? 1 : -1, syw = vc > T(0) ? BW : -BW;
        const bool zpos = wc > T(0);
        const size_t cell = (size_t)k * plane + (size_t)j * g.nx + i;
        const bool wr = active && EVP_DBG_OK(cell < plane * (size_t)g.nz);   // this cell's outputs are written
        const T* Bk = sm.B[k & 1][0];
        const T vx_ = fabs(uc) * g.idx, vy_ = fabs(vc) * g.idy, vz_ = fabs(wc) * g.idz;
        // ring offsets of the z stencil of this cell, far upwind first: planes
        // k-3 .. k+2 for a positive w, mirrored (k+3 .. k-2) otherwise
        int zo[6];
#pragma unroll
        for (int n = 0; n < 6; ++n) zo[n] = ((zpos ? k - 3 + n : k + 3 - n) & 7) * (6 * NT) + tid;
        T bn[6], advc[6];
        if constexpr (sizeof(T) == 4) {
            // single precision: the components in pairs (xx, xy), (xz, yy), (yz, zz),
            // which share the upwind side and |u|/h, on the packed f32x2 instructions
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const float* P0 = Bk + (2 * p) * BPL;
                const float* P1 = P0 + BPL;
                auto at = [&](int off) { return make_float2(P0[ob + off], P1[ob + off]); };
                auto zz = [&](int n) { return make_float2(Nf[zo[n] + (2 * p) * NT], Nf[zo[n] + (2 * p + 1) * NT]); };
                float2 s = upwind_term2(splat2(vx_), at(-3 * sx), at(-2 * sx), at(-sx), at(0), at(sx), at(2 * sx));
                s = add2(s, upwind_term2(splat2(vy_), at(-3 * syw), at(-2 * syw), at(-syw), at(0), at(syw), at(2 * syw)));
                // z stencil from the ring
                s = add2(s, upwind_term2(splat2(vz_), zz(0), zz(1), zz(2), zz(3), zz(4), zz(5)));
                advc[2 * p] = s.x;
                advc[2 * p + 1] = s.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const T* P = Bk + c * BPL;
                T adv = upwind_term(vx_, P[ob - 3 * sx], P[ob - 2 * sx], P[ob - sx], P[ob], P[ob + sx], P[ob + 2 * sx]);
                adv += upwind_term(vy_, P[ob - 3 * syw], P[ob - 2 * syw], P[ob - syw], P[ob], P[ob + syw], P[ob + 2 * syw]);
                // z stencil from the ring
                advc[c] = adv + upwind_term(vz_, Nf[zo[0] + c * NT], Nf[zo[1] + c * NT], Nf[zo[2] + c * NT], b0[c],
                                            Nf[zo[4] + c * NT], Nf[zo[5] + c * NT]);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const T* P = Bk + c * BPL;
            const T adv = advc[c];
            const int ra = row_of(c), cb = col_of(c);
            T ucd = T(0);
#pragma unroll
            for (int q = 0; q < 3; ++q) ucd += L[ra][q] * b0[symi(q, cb)] + b0[symi(ra, q)] * L[cb][q];
            const bool diag = (c == 0 || c == 3 || c == 5);
            const T src = ((diag ? av : T(0)) - F * b0[c]) * inv_lam;
            T rt = src + ucd - adv;
            if (DIFF && kad != T(0)) {
                const T bc = b0[c];
                const T zm = sm.N[(k - 1) & 7][c][tid], zp = sm.N[(k + 1) & 7][c][tid];
                rt += kad * ((P[ob - 1] + P[ob + 1] - T(2) * bc) * (g.idx * g.idx)
                             + (P[ob - BW] + P[ob + BW] - T(2) * bc) * (g.idy * g.idy)
                             + (zm + zp - T(2) * bc) * (g.idz * g.idz));
            }
            if (RHS_ONLY) {
                if (wr) a.RT[c][cell] = rt;
            } else {
                T inc = dtz * rt;
                if (READ_H) inc += dtx * sm.H[k & 1][c][tid];
                bn[c] = b0[c] + inc;
                if (wr) {
                    a.Bn[c][cell] = bn[c];
                    if (WRITE_H) a.RT[c][cell] = rt;
                }
            }
        }
        if (wr && !RHS_ONLY) {
            // a non-finite component makes the sum non-finite
            if (!isfinite(bn[0] + bn[1] + bn[2] + bn[3] + bn[4] + bn[5])) bits |= EVP_BIT_NONFINITE;
            if (MODEL == EVP_FENE_P && bn[0] + bn[3] + bn[5] >= kL2) bits |= EVP_BIT_TRACE_LIMIT;
            const T det = bn[0] * (bn[3] * bn[5] - bn[4] * bn[4]) - bn[1] * (bn[1] * bn[5] - bn[4] * bn[2])
                          + bn[2] * (bn[1] * bn[4] - bn[3] * bn[2]);
            if (det < T(0)) bits |= EVP_BIT_DET_NEG;
            if (a.S[0]) {
                // summed polymer stress tau(B^k) + tau(B^{k-1}) of the cell (Table 1),
                // the divergence term of the momentum step
                const T gm = kgm;
                if (MODEL == EVP_FENE_P) {
                    const T Fo = kL2 / (kL2 - (b0[0] + b0[3] + b0[5]));
                    const T Fn = kL2 / (kL2 - (bn[0] + bn[3] + bn[5]));
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const bool d = (c == 0 || c == 3 || c == 5);
                        a.S[c][cell] = gm * (Fn * bn[c] - (d ? kaf : T(0))) + gm * (Fo * b0[c] - (d ? kaf : T(0)));
                    }
                } else if (MODEL == EVP_NEO_HOOKEAN) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) a.S[c][cell] = gm * bn[c] + gm * b0[c];
                } else {
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        const bool d = (c == 0 || c == 3 || c == 5);
                        a.S[c][cell] = gm * (bn[c] - (d ? T(1) : T(0))) + gm * (b0[c] - (d ? T(1) : T(0)));
                    }
                }
            }
        }

        // ---- plane k+1 (halo) and ring slot k+4 have landed; after the barrier
        // they are visible to every thread
        cp_async_wait_all();
        __syncthreads();
    }
    if (bits) atomicOr(a.status, bits);
    EVP_DBG_REPORT(a.status);
}

template <typename T, int MODEL, int MODE, bool DIFF, bool VEC>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
k_stress(const Geo<T> g, const ModelConst mc, const StressArgs<T> a, int kz_chunk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    stress_tile<T, MODEL, MODE, DIFF, VEC>(g, mc, a, kz_chunk, blockIdx.x, blockIdx.y, blockIdx.z, smraw);
}

// Batched form: a persistent grid walks a work list of (member, tile x, tile y,
// z chunk) over the members of a batch, whose grids may differ; the members'
// arguments sit in the kernel's parameter space.
template <typename T, int MODEL, int MODE, bool DIFF, bool VEC>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
k_stress_batch(const __grid_constant__ StressBatch<T> p, const int4* __restrict__ work, int nwork) {
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int4 t = __ldg(work + w);
        const StressMember<T>& m = p.m[t.x];
        stress_tile<T, MODEL, MODE, DIFF, VEC>(m.g, m.mc, m.a, m.kz, t.y, t.z, t.w, smraw);
        __syncthreads();
    }
}

}  // namespace

template <typename T, bool VEC>
cudaError_t launch_stress_v(const Geo<T>& g, const ModelConst& mc, const StressArgs<T>& a, cudaStream_t st,
                            dim3 grid, int kz, bool pdl) {
    dim3 block(TX, TY, 1);
    const size_t smem = sizeof(StressSmem<T>);
    const int mode = a.rhs_only ? 0 : (!a.read_hist ? 1 : (a.write_hist ? 2 : 3));
    const int diff = mc.art_diff > 0.0 ? 1 : 0;
    switch ((mc.model * 4 + mode) * 2 + diff) {
#define EVP_LAUNCH_STRESS_D(M, MD, D)                                                                        \
    case (M * 4 + MD) * 2 + D:                                                                               \
        cudaFuncSetAttribute(k_stress<T, M, MD, D, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                             (int)smem);                                                                     \
        if (cudaError_t e = launch_k(k_stress<T, M, MD, D, VEC>, grid, block, smem, st, pdl, g, mc, a, kz))  \
            return e;                                                                                        \
        break;
#define EVP_LAUNCH_STRESS(M, MD) EVP_LAUNCH_STRESS_D(M, MD, false) EVP_LAUNCH_STRESS_D(M, MD, true)
        EVP_LAUNCH_STRESS(EVP_OLDROYD_B, 0)
        EVP_LAUNCH_STRESS(EVP_OLDROYD_B, 1)
        EVP_LAUNCH_STRESS(EVP_OLDROYD_B, 2)
        EVP_LAUNCH_STRESS(EVP_OLDROYD_B, 3)
        EVP_LAUNCH_STRESS(EVP_FENE_P, 0)
        EVP_LAUNCH_STRESS(EVP_FENE_P, 1)
        EVP_LAUNCH_STRESS(EVP_FENE_P, 2)
        EVP_LAUNCH_STRESS(EVP_FENE_P, 3)
        EVP_LAUNCH_STRESS(EVP_SARAMITO, 0)
        EVP_LAUNCH_STRESS(EVP_SARAMITO, 1)
        EVP_LAUNCH_STRESS(EVP_SARAMITO, 2)
        EVP_LAUNCH_STRESS(EVP_SARAMITO, 3)
        EVP_LAUNCH_STRESS(EVP_NEO_HOOKEAN, 0)
        EVP_LAUNCH_STRESS(EVP_NEO_HOOKEAN, 1)
        EVP_LAUNCH_STRESS(EVP_NEO_HOOKEAN, 2)
        EVP_LAUNCH_STRESS(EVP_NEO_HOOKEAN, 3)
#undef EVP_LAUNCH_STRESS
#undef EVP_LAUNCH_STRESS_D
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

// Batched stress update: one persistent launch over the work list (members of one
// model, one mode and one staging kind, the caller groups them so).
template <typename T>
cudaError_t launch_stress_batch(const StressBatch<T>& p, int model, int mode, bool vec, const int4* work, int nwork,
                                int ctas, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    dim3 block(TX, TY, 1);
    const size_t smem = sizeof(StressSmem<T>);
    const dim3 grid(ctas < nwork ? ctas : nwork);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch_k(kern, grid, block, smem, st, false, p, work, nwork);
    };
    switch ((model * 4 + mode) * 2 + (vec ? 1 : 0)) {
#define EVP_LAUNCH_STRESS_B(M, MD)                                            \
    case (M * 4 + MD) * 2 + 0: return go(k_stress_batch<T, M, MD, false, false>); \
    case (M * 4 + MD) * 2 + 1: return go(k_stress_batch<T, M, MD, false, true>);
        EVP_LAUNCH_STRESS_B(EVP_OLDROYD_B, 1)
        EVP_LAUNCH_STRESS_B(EVP_OLDROYD_B, 2)
        EVP_LAUNCH_STRESS_B(EVP_OLDROYD_B, 3)
        EVP_LAUNCH_STRESS_B(EVP_FENE_P, 1)
        EVP_LAUNCH_STRESS_B(EVP_FENE_P, 2)
        EVP_LAUNCH_STRESS_B(EVP_FENE_P, 3)
        EVP_LAUNCH_STRESS_B(EVP_SARAMITO, 1)
        EVP_LAUNCH_STRESS_B(EVP_SARAMITO, 2)
        EVP_LAUNCH_STRESS_B(EVP_SARAMITO, 3)
#undef EVP_LAUNCH_STRESS_B
        default: return cudaErrorInvalidValue;
    }
}

// resident CTAs of the stress kernel per SM (shared memory and registers)
template <typename T>
int stress_ctas_per_sm() { return sizeof(T) == 4 ? 2 : 1; }

template <typename T>
cudaError_t launch_stress(const Geo<T>& g, const ModelConst& mc, const StressArgs<T>& a,
                          cudaStream_t st, const TimingHook& th) {
    // z chunks: about four waves of CTAs over all SMs (two CTAs per SM in FP32,
    // one in FP64); small grids go down to one plane per CTA so that every SM works
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    const int per_sm = sizeof(T) == 4 ? 2 : 1;
    int chunks = (4 * 152 * per_sm + tiles - 1) / tiles;
    chunks = chunks > g.nz ? g.nz : chunks;
    const int kz = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + kz - 1) / kz;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, chunks);
    th.b(K_STRESS);
    cudaError_t e;
    // 16-byte chunks need whole chunks per row: always so in FP64 (nx is even)
    if constexpr (sizeof(T) == 8) {
        e = launch_stress_v<T, true>(g, mc, a, st, grid, kz, th.pdl);
    } else {
        e = (g.nx * sizeof(T)) % 16 == 0 ? launch_stress_v<T, true>(g, mc, a, st, grid, kz, th.pdl)
                                         : launch_stress_v<T, false>(g, mc, a, st, grid, kz, th.pdl);
    }
    if (e != cudaSuccess) return e;
    th.e(K_STRESS);
    return cudaGetLastError();
}


}  // namespace evp
