// Device self-test of the integer-operation conversions between binary32 and
// binary64 (widen_f32, narrow_f64) against the conversion instructions: bit for
// bit, except that binary32-subnormal values must come out as the signed zero and
// a NaN as some NaN.
#include <algorithm>

#include "evp_internal.cuh"

namespace evp {

namespace {

// Plain (non-tensor) FMA throughput: every thread runs NACC independent chains of
// ``iters`` fused multiply-adds acc = acc * m + c with run-time m and c, so that
// nothing folds and each chain keeps the pipe busy at full occupancy.  Single
// precision uses the packed f32x2 instruction (two lanes per instruction), the
// form the stress kernel issues.  A result equal to ``never`` would be stored, so
// the chains cannot be removed.
constexpr int NACC = 8;

__global__ void __launch_bounds__(256) k_peak_f32(float* out, int iters, float m, float c, float never) {
    float2 acc[NACC];
#pragma unroll
    for (int q = 0; q < NACC; ++q) acc[q] = make_float2(threadIdx.x * 1e-3f + q, q * 0.5f);
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < NACC; ++q) acc[q] = __ffma2_rn(acc[q], m2, c2);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < NACC; ++q) s += acc[q].x + acc[q].y;
    if (s == never) out[0] = s;
}

__global__ void __launch_bounds__(256) k_peak_f64(double* out, int iters, double m, double c, double never) {
    double acc[NACC];
#pragma unroll
    for (int q = 0; q < NACC; ++q) acc[q] = threadIdx.x * 1e-3 + q;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < NACC; ++q) acc[q] = fma(acc[q], m, c);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < NACC; ++q) s += acc[q];
    if (s == never) out[0] = s;
}

}  // namespace

cudaError_t run_fma_peak(int precision, double* flops) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    void* d = nullptr;
    e = cudaMalloc(&d, 16);
    if (e != cudaSuccess) return e;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int threads = 256, blocks = sms * 8;
    // about 20-40 ms per launch at the expected rates (80 TFLOP/s FP32, ~1.3 FP64)
    const int iters = precision == EVP_FP32 ? 65536 : 2048;
    const double per_launch = 2.0 * NACC * (precision == EVP_FP32 ? 2.0 : 1.0) * iters * double(threads) * blocks;
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a);
        if (precision == EVP_FP32)
            k_peak_f32<<<blocks, threads>>>(static_cast<float*>(d), iters, 0.999999f, 1e-7f, -1.2345e30f);
        else
            k_peak_f64<<<blocks, threads>>>(static_cast<double*>(d), iters, 0.999999999, 1e-12, -1.2345e300);
        cudaEventRecord(b);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        // the first launch is a warm-up
        if (e == cudaSuccess && rep > 0 && ms > 0.f) best = std::max(best, per_launch / (ms * 1e-3));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(d);
    *flops = best;
    return e;
}

namespace {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): counter -> 64 well-mixed bits
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// every binary32 bit pattern exactly once: thread t takes patterns t*per .. t*per+per-1
__global__ void k_selftest_widen(unsigned long long* bad, unsigned per) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long local = 0;
    for (unsigned q = 0; q < per; ++q) {
        const unsigned b = (unsigned)(t * per + q);
        const float x = __uint_as_float(b);
        const double got = widen_f32(x);
        const unsigned e = (b >> 23) & 0xffu;
        bool ok;
        if (e == 0u) ok = __double_as_longlong(got) == (long long)((unsigned long long)(b & 0x80000000u) << 32);
        else if (x != x) ok = got != got;
        else ok = __double_as_longlong(got) == __double_as_longlong((double)x);
        if (!ok) ++local;
    }
    if (local) atomicAdd(bad, local);
}

// binary64 patterns: exponents 880..1170 (both ends of the normal float range)
// with random fractions, the rounding ties and their neighbours, and one pattern
// in sixteen with an arbitrary exponent (zero, subnormals, infinities, NaN)
__global__ void k_selftest_narrow(unsigned long long* bad, unsigned per) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long local = 0;
    for (unsigned q = 0; q < per; ++q) {
        const unsigned long long id = t * per + q;
        const unsigned long long r1 = splitmix64(2 * id), r2 = splitmix64(2 * id + 1);
        unsigned long long e = 880ull + (r2 % 291ull);
        if (((r2 >> 40) & 15ull) == 0ull) e = (r2 >> 20) & 0x7ffull;
        unsigned long long frac = r1 & 0xfffffffffffffull;
        const long long kind = (long long)((r2 >> 50) & 3ull);
        // kinds 1..3: the low 29 bits one below the tie, at it, one above it
        if (kind) frac = (frac & ~0x1fffffffull) | (unsigned long long)(0x10000000ll + kind - 2);
        const unsigned long long b = (r1 & 0x8000000000000000ull) | (e << 52) | frac;
        const double x = __longlong_as_double((long long)b);
        const float got = narrow_f64(x), ref = (float)x;
        const unsigned rb = __float_as_uint(ref);
        bool ok;
        if (x != x) ok = got != got;
        else if (e < 897ull) ok = __float_as_uint(got) == (rb & 0x80000000u);   // |x| < 2^-126: signed zero
        else ok = __float_as_uint(got) == rb;
        if (!ok) ++local;
    }
    if (local) atomicAdd(bad, local);
}

}  // namespace

cudaError_t run_selftest(unsigned long long* mismatches) {
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
    const unsigned per = 1024, threads = 256;
    const unsigned long long widen_threads = (1ull << 32) / per;             // 4 Mi threads: 2^32 patterns
    const unsigned narrow_blocks = 4096;                                      // 2^30 patterns
    if (e == cudaSuccess) {
        k_selftest_widen<<<(unsigned)(widen_threads / threads), threads>>>(d, per);
        k_selftest_narrow<<<narrow_blocks, threads>>>(d + 1, per);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    *mismatches = h[0] + h[1];
    return e;
}

}  // namespace evp
