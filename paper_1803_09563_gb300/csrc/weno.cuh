// Fifth-order WENO (Sec. 3.1) used by the stress and level-set kernels.
#pragma once

#include <cfloat>

namespace evp {

// Fifth-order WENO combination (Sec. 3.1) of five undivided differences ordered
// from far upwind to downwind, times ``scale``: Jiang-Shu smoothness indicators,
// linear weights (1/10, 6/10, 3/10), eps = 1e-6, power 2.  Algebraically
// rearranged for fewer operations, with the same value:
//  * the indicators use the second differences a_k and b_k of the differences;
//    eps and all three indicators are scaled by 12/13 (a common factor of
//    eps + S_k cancels in the normalised weights);
//  * in double precision the weights alpha_k = d_k/e_k^2 are multiplied through by
//    10 e_1^2 e_2^2 e_3^2, which leaves one division;
//  * in single precision those products could overflow, so the weights are formed
//    from three approximate reciprocals of the squared indicators (no branch; an
//    indicator beyond ~1e19 gets a zero weight).
// Approximate single-precision reciprocal (PTX rcp.approx.ftz.f32, about one ulp;
// a subnormal result flushes to zero, 1/inf = 0).  The WENO weights below use it
// directly: their operands are at least the squared epsilon term (~8.5e-13) or
// overflowed indicators, which should get weight zero anyway, so the operand range
// handling of the general fast division is not needed.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename T>
__device__ __forceinline__ T weno5(T v1, T v2, T v3, T v4, T v5, T scale) {
    const T eps = T(1.0e-6 * 12.0 / 13.0), r = T(3.0 / 13.0);
    // candidates: q1, 6 q2, 3 q3
    const T q1 = v1 * T(1.0 / 3.0) - v2 * T(7.0 / 6.0) + v3 * T(11.0 / 6.0);
    const T q2 = -v2 + T(5) * v3 + T(2) * v4;
    const T q3 = v3 + T(2.5) * v4 - T(0.5) * v5;
    const T e12 = v1 - v2, e23 = v2 - v3, e34 = v3 - v4, e45 = v4 - v5;
    const T a1 = e12 - e23, a2 = e23 - e34, a3 = e34 - e45;
    const T b1 = a1 - T(2) * e23, b2 = e23 + e34, b3 = a3 + T(2) * e34;
    // (12/13)(eps + S_k) = a_k^2 + (3/13) b_k^2 + (12/13) eps
    T s1 = fma(b1 * r, b1, fma(a1, a1, eps));
    T s2 = fma(b2 * r, b2, fma(a2, a2, eps));
    T s3 = fma(b3 * r, b3, fma(a3, a3, eps));
    s1 *= s1;
    s2 *= s2;
    s3 *= s3;
    if (sizeof(T) == 4) {
        const float x1 = rcp_approx(float(s1)), x2 = rcp_approx(float(s2)), x3 = rcp_approx(float(s3));
        const float num = fmaf(x3, float(q3), fmaf(x2, float(q2), x1 * float(q1))) * float(scale);
        const float den = fmaf(3.0f, x3, fmaf(6.0f, x2, x1));
        return T(num * rcp_approx(den));
    }
    const T w1 = s2 * s3, w2 = s1 * s3, w3 = s1 * s2;
    const T den = fma(T(3), w3, fma(T(6), w2, w1));
    const T num = fma(w3, q3, fma(w2, q2, w1 * q1)) * scale;
    return num / den;
}

// Packed single-precision pairs (Blackwell f32x2 add / mul / fma: one instruction
// for both lanes, each lane rounded exactly as the scalar instruction).
__device__ __forceinline__ float2 splat2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }

// weno5<float> on two independent stencils at once (the lanes of each argument),
// with the same operations in the same order.
__device__ __forceinline__ float2 weno5x2(float2 v1, float2 v2, float2 v3, float2 v4, float2 v5, float2 scale) {
    const float2 eps = splat2(float(1.0e-6 * 12.0 / 13.0)), r = splat2(float(3.0 / 13.0));
    const float2 q1 = fma2(v3, splat2(float(11.0 / 6.0)), fma2(v2, splat2(float(-7.0 / 6.0)), mul2(v1, splat2(float(1.0 / 3.0)))));
    const float2 q2 = fma2(v4, splat2(2.0f), fma2(v3, splat2(5.0f), neg2(v2)));
    const float2 q3 = fma2(v5, splat2(-0.5f), fma2(v4, splat2(2.5f), v3));
    const float2 e12 = sub2(v1, v2), e23 = sub2(v2, v3), e34 = sub2(v3, v4), e45 = sub2(v4, v5);
    const float2 a1 = sub2(e12, e23), a2 = sub2(e23, e34), a3 = sub2(e34, e45);
    const float2 b1 = fma2(e23, splat2(-2.0f), a1), b2 = add2(e23, e34), b3 = fma2(e34, splat2(2.0f), a3);
    float2 s1 = fma2(mul2(b1, r), b1, fma2(a1, a1, eps));
    float2 s2 = fma2(mul2(b2, r), b2, fma2(a2, a2, eps));
    float2 s3 = fma2(mul2(b3, r), b3, fma2(a3, a3, eps));
    s1 = mul2(s1, s1);
    s2 = mul2(s2, s2);
    s3 = mul2(s3, s3);
    const float2 x1 = rcp2(s1), x2 = rcp2(s2), x3 = rcp2(s3);
    const float2 num = mul2(fma2(x3, q3, fma2(x2, q2, mul2(x1, q1))), scale);
    const float2 den = fma2(splat2(3.0f), x3, fma2(splat2(6.0f), x2, x1));
    return mul2(num, rcp2(den));
}

// upwind_term on two stencils at once.
__device__ __forceinline__ float2 upwind_term2(float2 vih, float2 pm3, float2 pm2, float2 pm1, float2 p0, float2 pp1,
                                               float2 pp2) {
    return weno5x2(sub2(pm2, pm3), sub2(pm1, pm2), sub2(p0, pm1), sub2(pp1, p0), sub2(pp2, pp1), vih);
}

// |u| * (upwind WENO5 derivative) of a centred field along one axis, from the
// six values phi(c + m*sig*step), m = -3..2, where sig = +1 for a positive
// velocity (left-biased stencil) and -1 otherwise (right-biased, mirrored; the
// differences then change sign exactly, and so does the WENO combination).
// ``vih`` = |u| / h.
template <typename T>
__device__ __forceinline__ T upwind_term(T vih, T pm3, T pm2, T pm1, T p0, T pp1, T pp2) {
    return weno5(pm2 - pm3, pm1 - pm2, p0 - pm1, pp1 - p0, pp2 - pp1, vih);
}

}  // namespace evp
