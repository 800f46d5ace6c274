// Device self-test of the integer-pipe binary32 -> binary64 widening (widen_f32)
// against the conversion instruction, bit for bit, over every binary32 pattern.
#include "evp_internal.cuh"

namespace evp {

namespace {

// every binary32 bit pattern exactly once: thread t takes patterns t*per .. t*per+per-1
__global__ void k_selftest_widen(unsigned long long* bad, unsigned per) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long local = 0;
    for (unsigned q = 0; q < per; ++q) {
        const unsigned b = (unsigned)(t * per + q);
        const float x = __uint_as_float(b);
        if (__double_as_longlong(widen_f32(x)) != __double_as_longlong((double)x)) ++local;
    }
    if (local) atomicAdd(bad, local);
}

}  // namespace

cudaError_t run_selftest(unsigned long long* mismatches) {
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    e = cudaMemset(d, 0, sizeof(unsigned long long));
    const unsigned per = 1024, threads = 256;
    const unsigned long long total_threads = (1ull << 32) / per;             // 4 Mi threads
    if (e == cudaSuccess) {
        k_selftest_widen<<<(unsigned)(total_threads / threads), threads>>>(d, per);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    *mismatches = h;
    return e;
}

}  // namespace evp
