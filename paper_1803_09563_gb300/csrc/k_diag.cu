// Monitoring reductions of evp_diagnostics: kinetic energy, det B and tr B, the
// cells the Saramito closure of Table 1 leaves yielded (F > 0), and non-finite
// cells, all in FP64 on the stored values.
//
//   k_diag        one (32 x 8 patch, z plane) work item after another per block
//                 (grid-stride over all items), one partial record per block
//   k_diag_final  one block folds the partial records in index order
//
// Both reductions run in a fixed order (thread-local sums, then a fixed shuffle
// tree, then the warps in index order, then the blocks in index order), so a
// repeated call on the same fields returns the same bits.  Not on the step's
// path: a monitoring call, HBM-bound (9 words a cell).
#include "evp_internal.cuh"

namespace evp {

namespace {

struct Acc {
    double ke, dmin, tmax;
    unsigned long long yielded, bad;
};

__device__ __forceinline__ void fold(Acc& a, const Acc& b) {
    a.ke += b.ke;
    a.dmin = fmin(a.dmin, b.dmin);   // fmin/fmax skip a NaN operand
    a.tmax = fmax(a.tmax, b.tmax);
    a.yielded += b.yielded;
    a.bad += b.bad;
}

__device__ __forceinline__ Acc shfl(const Acc& a, int o) {
    Acc r;
    r.ke = __shfl_xor_sync(0xffffffffu, a.ke, o);
    r.dmin = __shfl_xor_sync(0xffffffffu, a.dmin, o);
    r.tmax = __shfl_xor_sync(0xffffffffu, a.tmax, o);
    r.yielded = __shfl_xor_sync(0xffffffffu, a.yielded, o);
    r.bad = __shfl_xor_sync(0xffffffffu, a.bad, o);
    return r;
}

// Fold the block's 256 accumulators; thread 0 returns the result.
__device__ __forceinline__ Acc block_fold(Acc a) {
    __shared__ Acc red[8];
    const int t = threadIdx.y * blockDim.x + threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fold(a, shfl(a, o));
    if (lane == 0) red[warp] = a;
    __syncthreads();
    if (t == 0) {
        a = red[0];
        for (int q = 1; q < 8; ++q) fold(a, red[q]);
    }
    return a;
}

__device__ __forceinline__ Acc acc_zero() {
    Acc a;
    a.ke = 0.0;
    a.dmin = __longlong_as_double(0x7ff0000000000000ll);    // +inf
    a.tmax = __longlong_as_double((long long)0xfff0000000000000ull);   // -inf
    a.yielded = 0ull;
    a.bad = 0ull;
    return a;
}

// det of the symmetric B (xx, xy, xz, yy, yz, zz) by cofactor expansion along the
// first row; each product and sum rounded in the written order (no contraction)
__device__ __forceinline__ double det_sym(const double b[6]) {
    const double c0 = __dsub_rn(__dmul_rn(b[3], b[5]), __dmul_rn(b[4], b[4]));
    const double c1 = __dsub_rn(__dmul_rn(b[1], b[5]), __dmul_rn(b[4], b[2]));
    const double c2 = __dsub_rn(__dmul_rn(b[1], b[4]), __dmul_rn(b[3], b[2]));
    return __dadd_rn(__dsub_rn(__dmul_rn(b[0], c0), __dmul_rn(b[1], c1)), __dmul_rn(b[2], c2));
}

// |tau^d| > tau_y for tau = gm (B - I), |tau^d|^2 = 1/2 tau^d_ij tau^d_ij (Table 1,
// Saramito row), rounded in the written order
__device__ __forceinline__ bool yielded_cell(const double b[6], double gm, double tau_y) {
    double t[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c] = __dmul_rn(gm, (c == 0 || c == 3 || c == 5) ? __dsub_rn(b[c], 1.0) : b[c]);
    const double tr3 = __ddiv_rn(__dadd_rn(__dadd_rn(t[0], t[3]), t[5]), 3.0);
    const double d0 = __dsub_rn(t[0], tr3), d3 = __dsub_rn(t[3], tr3), d5 = __dsub_rn(t[5], tr3);
    double m2 = __dmul_rn(0.5, __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d3, d3)), __dmul_rn(d5, d5)));
    m2 = __dadd_rn(m2, __dmul_rn(t[1], t[1]));
    m2 = __dadd_rn(m2, __dmul_rn(t[2], t[2]));
    m2 = __dadd_rn(m2, __dmul_rn(t[4], t[4]));
    return __dsqrt_rn(m2) > tau_y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_diag(const Geo<T> g, const DiagArgs<T> a, DiagPart* __restrict__ parts) {
    const int tx = (g.nx + 31) / 32;
    const long long tiles = (long long)tx * ((g.ny + 7) / 8);
    const long long items = tiles * g.nz;
    const size_t plane = (size_t)g.nx * g.ny;
    Acc acc = acc_zero();
    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const int t = (int)(w % tiles), k = (int)(w / tiles);
        const int i = (t % tx) * 32 + threadIdx.x, j = (t / tx) * 8 + threadIdx.y;
        if (i >= g.nx || j >= g.ny) continue;
        const size_t o = (size_t)k * plane + (size_t)j * g.nx + i;
        const double u = (double)__ldg(a.U + o), v = (double)__ldg(a.V + o), wv = (double)__ldg(a.W + o);
        bool bad = !isfinite(u) || !isfinite(v) || !isfinite(wv);
        acc.ke += u * u + v * v + wv * wv;
        if (a.B[0]) {
            double b[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                b[c] = (double)__ldg(a.B[c] + o);
                bad = bad || !isfinite(b[c]);
            }
            acc.dmin = fmin(acc.dmin, det_sym(b));
            acc.tmax = fmax(acc.tmax, __dadd_rn(__dadd_rn(b[0], b[3]), b[5]));
            bool y = a.yield_mode == 1;
            if (a.yield_mode == 2) {
                const double gm = a.H ? __dmul_rn(__dmul_rn(a.mp1, (double)__ldg(a.H + o)), a.inv_lam) : a.gm;
                y = a.tau_y == 0.0 || yielded_cell(b, gm, a.tau_y);
            }
            acc.yielded += y ? 1ull : 0ull;
        }
        acc.bad += bad ? 1ull : 0ull;
    }
    acc = block_fold(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        DiagPart p;
        p.ke = acc.ke;
        p.min_det = acc.dmin;
        p.max_tr = acc.tmax;
        p.yielded = acc.yielded;
        p.nonfinite = acc.bad;
        parts[blockIdx.x] = p;
    }
}

__global__ void __launch_bounds__(256) k_diag_final(const DiagPart* __restrict__ parts, int nparts,
                                                    DiagPart* __restrict__ out) {
    Acc acc = acc_zero();
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) {
        Acc b;
        b.ke = parts[q].ke;
        b.dmin = parts[q].min_det;
        b.tmax = parts[q].max_tr;
        b.yielded = parts[q].yielded;
        b.bad = parts[q].nonfinite;
        fold(acc, b);
    }
    acc = block_fold(acc);
    if (threadIdx.x == 0) {
        out->ke = acc.ke;
        out->min_det = acc.dmin;
        out->max_tr = acc.tmax;
        out->yielded = acc.yielded;
        out->nonfinite = acc.bad;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_diag(const Geo<T>& g, const DiagArgs<T>& a, DiagPart* parts, DiagPart* out, cudaStream_t st) {
    const long long items = (long long)((g.nx + 31) / 32) * ((g.ny + 7) / 8) * g.nz;
    const int nb = (int)(items < DIAG_BLOCKS ? items : DIAG_BLOCKS);
    k_diag<T><<<nb, dim3(32, 8, 1), 0, st>>>(g, a, parts);
    k_diag_final<<<1, 256, 0, st>>>(parts, nb, out);
    return cudaGetLastError();
}

template cudaError_t launch_diag<float>(const Geo<float>&, const DiagArgs<float>&, DiagPart*, DiagPart*, cudaStream_t);
template cudaError_t launch_diag<double>(const Geo<double>&, const DiagArgs<double>&, DiagPart*, DiagPart*,
                                         cudaStream_t);

}  // namespace evp
