// S1 + S2: centre velocity and velocity gradient, WENO5 advection of the six
// components of B, the Table 1 closure and the RK3 update of Eq. rk3tau.
//
// RT = (a I - F B)/lambda - (u.grad B - B.grad u - grad u^T.B)     (Eq. rt / RK-rt)
// B^k = B^{k-1} + dt (zeta^k RT^{k-1} + xi^k RT^{k-2})            (Eq. rk3tau)
//
// One thread per cell; neighbours are read through the read-only cache.
#include <cfloat>

#include "evp_internal.cuh"

namespace evp {

namespace {

// Fifth-order WENO combination (Sec. 3.1) of five undivided differences ordered
// from far upwind to downwind: Jiang-Shu smoothness indicators, linear weights
// (1/10, 6/10, 3/10), eps = 1e-6, power 2.  The normalised weights
// alpha_k / sum(alpha) are formed by multiplying every alpha_k = d_k/e_k through
// by e_1 e_2 e_3, which leaves one division per reconstruction.
template <typename T>
__device__ __forceinline__ T weno5(T v1, T v2, T v3, T v4, T v5) {
    const T c13 = T(13.0 / 12.0), q = T(0.25), eps = T(1.0e-6);
    T q1 = v1 * T(1.0 / 3.0) - v2 * T(7.0 / 6.0) + v3 * T(11.0 / 6.0);
    T q2 = -v2 * T(1.0 / 6.0) + v3 * T(5.0 / 6.0) + v4 * T(1.0 / 3.0);
    T q3 = v3 * T(1.0 / 3.0) + v4 * T(5.0 / 6.0) - v5 * T(1.0 / 6.0);
    T a = v1 - T(2) * v2 + v3, b = v1 - T(4) * v2 + T(3) * v3;
    T s1 = c13 * a * a + q * b * b;
    a = v2 - T(2) * v3 + v4;
    b = v2 - v4;
    T s2 = c13 * a * a + q * b * b;
    a = v3 - T(2) * v4 + v5;
    b = T(3) * v3 - T(4) * v4 + v5;
    T s3 = c13 * a * a + q * b * b;
    T e1 = eps + s1, e2 = eps + s2, e3 = eps + s3;
    e1 *= e1;
    e2 *= e2;
    e3 *= e3;
    T w1 = T(0.1) * e2 * e3, w2 = T(0.6) * e1 * e3, w3 = T(0.3) * e1 * e2;
    T den = w1 + w2 + w3;
    if (sizeof(T) == 4 && !(den <= T(FLT_MAX))) {
        // products overflowed single precision: fall back to the three-division form
        w1 = T(0.1) / e1;
        w2 = T(0.6) / e2;
        w3 = T(0.3) / e3;
        den = w1 + w2 + w3;
    }
    return (w1 * q1 + w2 * q2 + w3 * q3) / den;
}

// storage index of the symmetric component (a, b): xx xy xz yy yz zz
__device__ __forceinline__ constexpr int symi(int a, int b) {
    return a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5));
}
__device__ __forceinline__ constexpr int row_of(int c) { return c < 3 ? 0 : (c < 5 ? 1 : 2); }
__device__ __forceinline__ constexpr int col_of(int c) { return c == 0 ? 0 : ((c == 1 || c == 3) ? 1 : 2); }

// |u| * (upwind WENO5 derivative) of a centred field along one axis, from the
// six values phi(c + m*sig*step), m = -3..2, where sig = +1 for a positive
// velocity (left-biased stencil) and -1 otherwise (right-biased, mirrored).
template <typename T>
__device__ __forceinline__ T upwind_term(T vel, T ih, T pm3, T pm2, T pm1, T p0, T pp1, T pp2) {
    return fabs(vel) * ih * weno5(pm2 - pm3, pm1 - pm2, p0 - pm1, pp1 - p0, pp2 - pp1);
}

template <typename T, int MODEL>
__global__ void __launch_bounds__(256)
k_stress(const Geo<T> g, const ModelConst mc, const StressArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c0 = lin(g, i, j, k);
    const int im = wrap(i - 1, g.nx), km = wrap(k - 1, g.nz);

    // ---- S1: centre velocity and velocity gradient (Reading 5)
    const T Uc = __ldg(a.U + c0), Um = ld_uw(g, a.U, im, j, k);
    const T Vc = __ldg(a.V + c0), Vm = ld_v(g, a.V, i, j - 1, k);
    const T Wc = __ldg(a.W + c0), Wm = ld_uw(g, a.W, i, j, km);
    const T uc = T(0.5) * (Um + Uc), vc = T(0.5) * (Vm + Vc), wc = T(0.5) * (Wm + Wc);
    T L[3][3];
    L[0][0] = (Uc - Um) * g.idx;
    L[1][1] = (Vc - Vm) * g.idy;
    L[2][2] = (Wc - Wm) * g.idz;
    {
        // u centred: average of faces i-1 and i, odd ghosts in y at walls
        auto ucen = [&](int jj, int kk) {
            return T(0.5) * (ld_uw(g, a.U, i - 1, jj, kk) + ld_uw(g, a.U, i, jj, kk));
        };
        auto wcen = [&](int ii, int jj) {
            return T(0.5) * (ld_uw(g, a.W, ii, jj, k - 1) + ld_uw(g, a.W, ii, jj, k));
        };
        auto vcen = [&](int ii, int kk) {
            return T(0.5) * (ld_v(g, a.V, ii, j - 1, kk) + ld_v(g, a.V, ii, j, kk));
        };
        const T hx = T(0.5) * g.idx, hy = T(0.5) * g.idy, hz = T(0.5) * g.idz;
        L[0][1] = (ucen(j + 1, k) - ucen(j - 1, k)) * hy;
        L[0][2] = (ucen(j, k + 1) - ucen(j, k - 1)) * hz;
        L[1][0] = (vcen(i + 1, k) - vcen(i - 1, k)) * hx;
        L[1][2] = (vcen(i, k + 1) - vcen(i, k - 1)) * hz;
        L[2][0] = (wcen(i + 1, j) - wcen(i - 1, j)) * hx;
        L[2][1] = (wcen(i, j + 1) - wcen(i, j - 1)) * hy;
    }

    // ---- B at the cell and the Table 1 closure
    T b[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) b[c] = __ldg(a.B[c] + c0);
    T F = T(1), av = T(1);
    if (MODEL == EVP_FENE_P) {
        const T tr = b[0] + b[3] + b[5];
        F = T(mc.L2) / (T(mc.L2) - tr);
        av = T(mc.a_fene);
    } else if (MODEL == EVP_SARAMITO) {
        const T gm = T(mc.gmod);
        T t[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) t[c] = gm * (b[c] - ((c == 0 || c == 3 || c == 5) ? T(1) : T(0)));
        const T tr3 = (t[0] + t[3] + t[5]) / T(3);
        const T d0 = t[0] - tr3, d3 = t[3] - tr3, d5 = t[5] - tr3;
        const T mag = sqrt(T(0.5) * (d0 * d0 + d3 * d3 + d5 * d5) + t[1] * t[1] + t[2] * t[2] + t[4] * t[4]);
        const T ty = T(mc.tau_y);
        if (mag > T(0)) {
            const T f = T(1) - ty / mag;
            F = f > T(0) ? f : T(0);
        } else {
            F = ty > T(0) ? T(0) : T(1);
        }
        av = F;
    }

    // ---- per-direction stencil offsets: sig = +1 (left-biased) if velocity > 0
    const int sx = uc > T(0) ? 1 : -1, sy = vc > T(0) ? 1 : -1, sz = wc > T(0) ? 1 : -1;
    int xi_[6], yj_[6], zk_[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        xi_[m] = wrap(i + (m - 3) * sx, g.nx);
        yj_[m] = ycen(g, j + (m - 3) * sy);
        zk_[m] = wrap(k + (m - 3) * sz, g.nz);
    }
    const size_t rowk = (size_t)k * g.ny;

    const T inv_lam = T(mc.inv_lam);
    const T dtz = a.dt_zeta, dtx = a.dt_xi;
    unsigned bits = 0;
    T bn[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const T* __restrict__ Bc = a.B[c];
        // x
        T px[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) px[m] = __ldg(Bc + (rowk + j) * g.nx + xi_[m]);
        T adv = upwind_term(uc, g.idx, px[0], px[1], px[2], px[3], px[4], px[5]);
#pragma unroll
        for (int m = 0; m < 6; ++m) px[m] = __ldg(Bc + (rowk + yj_[m]) * g.nx + i);
        adv += upwind_term(vc, g.idy, px[0], px[1], px[2], px[3], px[4], px[5]);
#pragma unroll
        for (int m = 0; m < 6; ++m) px[m] = __ldg(Bc + ((size_t)zk_[m] * g.ny + j) * g.nx + i);
        adv += upwind_term(wc, g.idz, px[0], px[1], px[2], px[3], px[4], px[5]);

        // upper-convected terms (L B + B L^T)_ab, Reading 2
        const int ra = row_of(c), cb = col_of(c);
        T ucd = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) ucd += L[ra][q] * b[symi(q, cb)] + b[symi(ra, q)] * L[cb][q];
        const bool diag = (c == 0 || c == 3 || c == 5);
        const T src = ((diag ? av : T(0)) - F * b[c]) * inv_lam;
        const T rt = src + ucd - adv;

        if (a.rhs_only) {
            a.RT[c][c0] = rt;
        } else {
            T inc = dtz * rt;
            if (a.read_hist) inc += dtx * a.RT[c][c0];
            bn[c] = b[c] + inc;
            a.Bn[c][c0] = bn[c];
            if (a.write_hist) a.RT[c][c0] = rt;
            if (!isfinite(bn[c])) bits |= EVP_BIT_NONFINITE;
        }
    }
    if (!a.rhs_only) {
        if (MODEL == EVP_FENE_P && bn[0] + bn[3] + bn[5] >= T(mc.L2)) bits |= EVP_BIT_TRACE_LIMIT;
        const T det = bn[0] * (bn[3] * bn[5] - bn[4] * bn[4]) - bn[1] * (bn[1] * bn[5] - bn[4] * bn[2])
                      + bn[2] * (bn[1] * bn[4] - bn[3] * bn[2]);
        if (det < T(0)) bits |= EVP_BIT_DET_NEG;
        if (bits) atomicOr(a.status, bits);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_stress(const Geo<T>& g, const ModelConst& mc, const StressArgs<T>& a,
                          cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_STRESS);
    switch (mc.model) {
        case EVP_OLDROYD_B: k_stress<T, EVP_OLDROYD_B><<<grid, block, 0, st>>>(g, mc, a); break;
        case EVP_FENE_P: k_stress<T, EVP_FENE_P><<<grid, block, 0, st>>>(g, mc, a); break;
        case EVP_SARAMITO: k_stress<T, EVP_SARAMITO><<<grid, block, 0, st>>>(g, mc, a); break;
        default: return cudaErrorInvalidValue;
    }
    th.e(K_STRESS);
    return cudaGetLastError();
}

template cudaError_t launch_stress<float>(const Geo<float>&, const ModelConst&, const StressArgs<float>&,
                                          cudaStream_t, const TimingHook&);
template cudaError_t launch_stress<double>(const Geo<double>&, const ModelConst&, const StressArgs<double>&,
                                           cudaStream_t, const TimingHook&);

}  // namespace evp
