// S4-S8: the fast Poisson solver and projection of Eqs. NS-num2 and NS-num3.
//
//   lap(psi) = div(u*) / (2 alpha^k dt);  u^k = u* - 2 alpha^k dt grad(psi);  p^k = p^{k-1} + psi
//
// psi is found with FFTs in the periodic directions and, along a wall-bounded y,
// a tridiagonal (Thomas) solve per Fourier mode (FP64, or double-single in FP32
// states); the modal eigenvalues are
// those of the discrete 7-point Laplacian, (2 - 2 cos(2 pi m/n))/h^2.
//
// Passes over the spectral buffer spec[nz][ny][nx/2+1] (complex):
//   k_div_fftx    divergence of u* (scaled) fused into the x real-to-complex FFT;
//                 two real lines are packed into one complex FFT and split after.
//   k_fft_col     forward complex FFT along z (columns of TK consecutive kx).
//   k_fft_col     periodic y: forward FFT along y, modal division, inverse FFT
//                 (one pass).
//   k_thomas      walls: Thomas sweep along y per (kx, kz), pivots from a table; FP64
//                 for FP64 states, double-single (pairs of floats) for FP32 states.
//   k_fft_col     inverse FFT along z.
//   k_ifftx       x complex-to-real inverse FFT -> psi.
//   k_correct     u = u* - c grad psi, p += psi (non-finite -> status).
//   k_div_residual  FP64 max |div u| of a stored velocity (run by evp_sync).
// For power-of-two lengths 16 .. 256 the x and column passes use the register-
// resident two-pass kernels (k_div_fftx_r, k_fft_col_r, k_ifftx_r); other lengths
// use the shared-memory kernels below.
//
// The shared-memory FFT is a Stockham auto-sort transform with radix-4, -3 and
// -2 stages (n = 2^a 3^b), twiddles read from a table exp(-2 pi i m/n).
#include <cfloat>

#include "evp_internal.cuh"

namespace evp {

namespace {

template <typename T>
using C = typename Cplx<T>::type;

template <typename T>
__device__ __forceinline__ C<T> mk(T x, T y) {
    C<T> r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename T>
__device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T, bool INV>
__device__ __forceinline__ C<T> twmul(C<T> a, C<T> w) {
    if (INV) w.y = -w.y;
    return mk<T>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ C<T> rot(C<T> a) { return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x); }

// One Stockham pass structure over ``nlines`` lines held in shared memory:
// element (line l, index m) at buf[l*ls + m*es].  Butterflies j are spread over
// (tj, nj) and lines over (tl, nl).  Returns the buffer holding the result.
template <typename T, bool INV>
__device__ C<T>* fft_smem(C<T>* a, C<T>* b, int n, const int* rad, int nst, const C<T>* __restrict__ tw,
                          int nlines, int es, int ls, int tj, int nj, int tl, int nl) {
    int Ns = 1;
    for (int s = 0; s < nst; ++s) {
        const int R = rad[s];
        const int nR = n / R;
        const int tws = n / (Ns * R);
        const bool pow2 = (Ns & (Ns - 1)) == 0;
        for (int jb = tj; jb < nR; jb += nj) {
            const int kk = pow2 ? (jb & (Ns - 1)) : jb % Ns;
            const int dbase = (jb - kk) * R + kk;
            const C<T> w1 = __ldg(tw + kk * tws);
            if (R == 4) {
                const C<T> w2 = __ldg(tw + 2 * kk * tws), w3 = __ldg(tw + 3 * kk * tws);
                for (int l = tl; l < nlines; l += nl) {
                    const C<T>* s0 = a + (size_t)l * ls;
                    C<T>* d0 = b + (size_t)l * ls;
                    C<T> x0 = s0[(jb) * es];
                    C<T> x1 = twmul<T, INV>(s0[(jb + nR) * es], w1);
                    C<T> x2 = twmul<T, INV>(s0[(jb + 2 * nR) * es], w2);
                    C<T> x3 = twmul<T, INV>(s0[(jb + 3 * nR) * es], w3);
                    const C<T> s02 = add<T>(x0, x2), d02 = sub<T>(x0, x2);
                    const C<T> s13 = add<T>(x1, x3), r13 = rot<T, INV>(sub<T>(x1, x3));
                    d0[(dbase) * es] = add<T>(s02, s13);
                    d0[(dbase + Ns) * es] = add<T>(d02, r13);
                    d0[(dbase + 2 * Ns) * es] = sub<T>(s02, s13);
                    d0[(dbase + 3 * Ns) * es] = sub<T>(d02, r13);
                }
            } else if (R == 3) {
                const C<T> w2 = __ldg(tw + 2 * kk * tws);
                const T h3 = T(0.86602540378443864676);   // sin(2 pi / 3)
                for (int l = tl; l < nlines; l += nl) {
                    const C<T>* s0 = a + (size_t)l * ls;
                    C<T>* d0 = b + (size_t)l * ls;
                    C<T> x0 = s0[(jb) * es];
                    C<T> x1 = twmul<T, INV>(s0[(jb + nR) * es], w1);
                    C<T> x2 = twmul<T, INV>(s0[(jb + 2 * nR) * es], w2);
                    const C<T> s = add<T>(x1, x2), d = sub<T>(x1, x2);
                    const C<T> m = mk<T>(x0.x - T(0.5) * s.x, x0.y - T(0.5) * s.y);
                    const C<T> r = rot<T, INV>(d);
                    const C<T> t = mk<T>(h3 * r.x, h3 * r.y);
                    d0[(dbase) * es] = add<T>(x0, s);
                    d0[(dbase + Ns) * es] = add<T>(m, t);
                    d0[(dbase + 2 * Ns) * es] = sub<T>(m, t);
                }
            } else {
                for (int l = tl; l < nlines; l += nl) {
                    const C<T>* s0 = a + (size_t)l * ls;
                    C<T>* d0 = b + (size_t)l * ls;
                    C<T> x0 = s0[(jb) * es];
                    C<T> x1 = twmul<T, INV>(s0[(jb + nR) * es], w1);
                    d0[(dbase) * es] = add<T>(x0, x1);
                    d0[(dbase + Ns) * es] = sub<T>(x0, x1);
                }
            }
        }
        __syncthreads();
        C<T>* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Rows that the divergence of real line L (= k*ny + j) reads: u*, v*, w* of the
// line itself, v* of the row below (null at a wall: the face below j = 0 carries
// v = 0) and w* of the plane below (periodic in z).
template <typename T>
struct DivRows {
    const T* u;
    const T* v;
    const T* vm;
    const T* w;
    const T* wm;
};
template <typename T>
__device__ __forceinline__ DivRows<T> div_rows(const Geo<T>& g, const PoissonArgs<T>& a, int L) {
    const int k = L / g.ny, j = L - k * g.ny;
    const size_t o = (size_t)L * g.nx;
    DivRows<T> r;
    r.u = a.Us + o;
    r.v = a.Vs + o;
    r.w = a.Ws + o;
    const int jm = j > 0 ? j - 1 : (g.walls ? -1 : g.ny - 1);
    r.vm = jm < 0 ? nullptr : a.Vs + ((size_t)k * g.ny + jm) * g.nx;
    const int km = k > 0 ? k - 1 : g.nz - 1;
    r.wm = a.Ws + ((size_t)km * g.ny + j) * g.nx;
    return r;
}
// r = div(u*) * rscale at x index i of the line whose rows are ``r``
template <typename T>
__device__ __forceinline__ T div_value(const Geo<T>& g, const PoissonArgs<T>& a, const DivRows<T>& r, int i) {
    const int im = i > 0 ? i - 1 : g.nx - 1;
    const T du = __ldg(r.u + i) - __ldg(r.u + im);
    const T dv = __ldg(r.v + i) - (r.vm ? __ldg(r.vm + i) : T(0));
    const T dw = __ldg(r.w + i) - __ldg(r.wm + i);
    return (du * g.idx + dv * g.idy + dw * g.idz) * a.rscale;
}

// S4 + S5(x): r = div(u*)/(2 alpha dt) fused into the x real-to-complex FFT.
template <typename T>
__device__ __forceinline__ void k_div_fftx_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a, int np) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx, nxh = nx / 2 + 1;
    C<T>* sa = reinterpret_cast<C<T>*>(smraw);
    C<T>* sb = sa + (size_t)np * nx;
    const int NL = g.ny * g.nz;
    const int q0 = blockIdx.x * np;
    for (int l = threadIdx.y; l < np; l += blockDim.y) {
        const int L0 = 2 * (q0 + l), L1 = L0 + 1;
        C<T>* dst = sa + (size_t)l * nx;
        if (a.rhs) {
            // explicit right-hand side (the plain Poisson solve)
            for (int i = threadIdx.x; i < nx; i += blockDim.x)
                dst[i] = mk<T>(L0 < NL ? __ldg(a.rhs + (size_t)L0 * nx + i) : T(0),
                               L1 < NL ? __ldg(a.rhs + (size_t)L1 * nx + i) : T(0));
            continue;
        }
        const bool ok0 = L0 < NL, ok1 = L1 < NL;
        const DivRows<T> r0 = div_rows(g, a, ok0 ? L0 : 0), r1 = div_rows(g, a, ok1 ? L1 : 0);
#pragma unroll 4
        for (int i = threadIdx.x; i < nx; i += blockDim.x)
            dst[i] = mk<T>(ok0 ? div_value(g, a, r0, i) : T(0), ok1 ? div_value(g, a, r1, i) : T(0));
    }
    __syncthreads();
    C<T>* res = fft_smem<T, false>(sa, sb, nx, tb.radx, tb.nrx, tb.twx, np, 1, nx, threadIdx.x, blockDim.x,
                                   threadIdx.y, blockDim.y);
    // split the packed pair: A_m = (Z_m + conj Z_{n-m})/2, B_m = (Z_m - conj Z_{n-m})/(2i)
    for (int l = threadIdx.y; l < np; l += blockDim.y) {
        const int L0 = 2 * (q0 + l), L1 = L0 + 1;
        if (L0 >= NL) continue;
        for (int m = threadIdx.x; m < nxh; m += blockDim.x) {
            const C<T> Z = res[(size_t)l * nx + m];
            const C<T> Zr = res[(size_t)l * nx + (m == 0 ? 0 : nx - m)];
            a.spec[(size_t)L0 * nxh + m] = mk<T>(T(0.5) * (Z.x + Zr.x), T(0.5) * (Z.y - Zr.y));
            if (L1 < NL) a.spec[(size_t)L1 * nxh + m] = mk<T>(T(0.5) * (Z.y + Zr.y), T(0.5) * (Zr.x - Z.x));
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(256)
k_div_fftx(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a, int np) {
    k_div_fftx_body<T>(g, tb, a, np);
}
template <typename T>
__global__ void __launch_bounds__(256)
k_div_fftx_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p, int np) {
    k_div_fftx_body<T>(g, tb, p.a[blockIdx.z], np);
}


// S7(x): complex-to-real inverse FFT along x of two lines per complex FFT -> psi
template <typename T>
__device__ __forceinline__ void k_ifftx_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a, int np) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx, nxh = nx / 2 + 1, half = nx / 2;
    C<T>* sa = reinterpret_cast<C<T>*>(smraw);
    C<T>* sb = sa + (size_t)np * nx;
    const int NL = g.ny * g.nz;
    const int q0 = blockIdx.x * np;
#pragma unroll 2
    for (int l = threadIdx.y; l < np; l += blockDim.y) {
        const int L0 = 2 * (q0 + l), L1 = L0 + 1;
#pragma unroll 4
        for (int m = threadIdx.x; m < nx; m += blockDim.x) {
            C<T> A = mk<T>(T(0), T(0)), B = mk<T>(T(0), T(0));
            const int mm = m <= half ? m : nx - m;
            if (L0 < NL) A = a.spec[(size_t)L0 * nxh + mm];
            if (L1 < NL) B = a.spec[(size_t)L1 * nxh + mm];
            if (mm == 0 || mm == half) {   // DC and Nyquist of a real line are real
                A.y = T(0);
                B.y = T(0);
            }
            if (m > half) {                // Hermitian extension
                A.y = -A.y;
                B.y = -B.y;
            }
            sa[(size_t)l * nx + m] = mk<T>(A.x - B.y, A.y + B.x);
        }
    }
    __syncthreads();
    C<T>* res = fft_smem<T, true>(sa, sb, nx, tb.radx, tb.nrx, tb.twx, np, 1, nx, threadIdx.x, blockDim.x,
                                  threadIdx.y, blockDim.y);
    for (int l = threadIdx.y; l < np; l += blockDim.y) {
        const int L0 = 2 * (q0 + l), L1 = L0 + 1;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const C<T> z = res[(size_t)l * nx + i];
            if (L0 < NL) a.psi[(size_t)L0 * nx + i] = z.x * a.out_scale;
            if (L1 < NL) a.psi[(size_t)L1 * nx + i] = z.y * a.out_scale;
        }
    }
}
template <typename T>
__global__ void __launch_bounds__(256)
k_ifftx(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a, int np) {
    k_ifftx_body<T>(g, tb, a, np);
}
template <typename T>
__global__ void __launch_bounds__(256)
k_ifftx_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p, int np) {
    k_ifftx_body<T>(g, tb, p.a[blockIdx.z], np);
}


// Column FFT along z (or y) over TK consecutive kx.  SOLVE (periodic y pass):
// forward FFT, multiply by -norm/(lx+ly+lz) (zero mode -> 0), inverse FFT.
template <typename T, bool INV, bool SOLVE>
__device__ __forceinline__ void k_fft_col_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a, int axis_y, size_t estride, size_t ostride, int tk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = axis_y ? g.ny : g.nz;
    const int* rad = axis_y ? tb.rady : tb.radz;
    const int nrad = axis_y ? tb.nry : tb.nrz;
    const C<T>* tw = axis_y ? tb.twy : tb.twz;
    C<T>* sa = reinterpret_cast<C<T>*>(smraw);
    C<T>* sb = sa + (size_t)n * tk;
    const int nxh = g.nx / 2 + 1;
    const int kx0 = blockIdx.x * tk;
    const size_t base = blockIdx.y * ostride;
#pragma unroll 8
    for (int m = threadIdx.y; m < n; m += blockDim.y)
        for (int t = threadIdx.x; t < tk; t += blockDim.x) {
            const int kx = kx0 + t;
            sa[(size_t)m * tk + t] = kx < nxh ? a.spec[base + m * estride + kx] : mk<T>(T(0), T(0));
        }
    __syncthreads();
    C<T>* res = fft_smem<T, INV>(sa, sb, n, rad, nrad, tw, tk, tk, 1, threadIdx.y, blockDim.y, threadIdx.x,
                                 blockDim.x);
    if (SOLVE) {
        const int kz = blockIdx.y;
        const T lz = __ldg(tb.lamz + kz);
        for (int m = threadIdx.y; m < n; m += blockDim.y)
            for (int t = threadIdx.x; t < tk; t += blockDim.x) {
                const int kx = kx0 + t;
                if (kx >= nxh) continue;
                const T lam = __ldg(tb.lamx + kx) + __ldg(tb.lamy + m) + lz;
                const T f = a.hcoef > T(0) ? T(a.norm) / (T(1) + a.hcoef * lam)
                                           : (lam == T(0) ? T(0) : T(-a.norm) / lam);
                C<T> v = res[(size_t)m * tk + t];
                res[(size_t)m * tk + t] = mk<T>(v.x * f, v.y * f);
            }
        __syncthreads();
        C<T>* other = (res == sa) ? sb : sa;
        res = fft_smem<T, true>(res, other, n, rad, nrad, tw, tk, tk, 1, threadIdx.y, blockDim.y, threadIdx.x,
                                blockDim.x);
    }
    for (int m = threadIdx.y; m < n; m += blockDim.y)
        for (int t = threadIdx.x; t < tk; t += blockDim.x) {
            const int kx = kx0 + t;
            if (kx < nxh) a.spec[base + m * estride + kx] = res[(size_t)m * tk + t];
        }
}
template <typename T, bool INV, bool SOLVE>
__global__ void __launch_bounds__(256)
k_fft_col(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a, int axis_y, size_t estride,
          size_t ostride, int tk) {
    k_fft_col_body<T, INV, SOLVE>(g, tb, a, axis_y, estride, ostride, tk);
}
template <typename T, bool INV, bool SOLVE>
__global__ void __launch_bounds__(256)
k_fft_col_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p, int axis_y, size_t estride, size_t ostride, int tk) {
    k_fft_col_body<T, INV, SOLVE>(g, tb, p.a[blockIdx.z], axis_y, estride, ostride, tk);
}


// ---- register-resident column FFTs for n = R1 * R2 (powers of two, n <= 256)
//
// Cooley-Tukey in two passes with one shared-memory exchange:
//   X[k1 + R1 k2] = sum_j2 W_R2^(j2 k2) W_n^(j2 k1) sum_j1 x[R2 j1 + j2] W_R1^(j1 k1)
// pass 1: one thread per (column, j2) takes the R1-point DFT over j1 in registers,
// multiplies by W_n^(j2 k1) and stores to shared memory; pass 2: one thread per
// (column, k1) takes the R2-point DFT over j2.  The inverse transform (conjugate
// twiddles) has the same structure.  Twiddles come from the table exp(-2 pi i m/n).

template <int R>
__device__ __forceinline__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// In-register R-point DFT (R a power of two), natural order in and out: radix-2
// decimation in time over the bit-reversed input.  tw[m * ts] = exp(-2 pi i m/R)
// (conjugated for INV).
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(C<T> (&x)[R], const C<T>* __restrict__ tw, int ts) {
    C<T> y[R];
#pragma unroll
    for (int i = 0; i < R; ++i) y[bitrev<R>(i)] = x[i];
#pragma unroll
    for (int h = 1; h < R; h *= 2) {
#pragma unroll
        for (int g0 = 0; g0 < R; g0 += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                const int m = k * (R / (2 * h));        // W_2h^k = W_R^m
                C<T> b = y[g0 + k + h];
                if (R >= 4 && m == R / 4) b = rot<T, INV>(b);   // W_R^(R/4) = -i
                else if (m != 0) b = twmul<T, INV>(b, __ldg(tw + m * ts));
                y[g0 + k + h] = sub<T>(y[g0 + k], b);
                y[g0 + k] = add<T>(y[g0 + k], b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] = y[i];
}

// Column FFT along z (or y) over tk consecutive kx, as k_fft_col, for n = R1 R2.
// Threads: (tk, max(R1, R2)).  SOLVE: forward, modal division, inverse (the
// inverse runs the two passes in reverse order, so its input is the forward
// output as each thread holds it).
template <typename T, bool INV, bool SOLVE, int R1, int R2>
__device__ __forceinline__ void k_fft_col_r_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a, int axis_y, size_t estride, size_t ostride, int tk) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    C<T>* Y = reinterpret_cast<C<T>*>(smraw);           // [R2][R1][tk]
    const C<T>* tw = axis_y ? tb.twy : tb.twz;
    const int nxh = g.nx / 2 + 1;
    const int t = threadIdx.x, q = threadIdx.y;
    const int kx = blockIdx.x * tk + t;
    const bool ok = kx < nxh;
    const size_t base = blockIdx.y * ostride + (ok ? kx : 0);
    if (q < R2) {
        C<T> x[R1];
#pragma unroll
        for (int j1 = 0; j1 < R1; ++j1)
            x[j1] = ok ? a.spec[base + (size_t)(R2 * j1 + q) * estride] : mk<T>(T(0), T(0));
        dft_reg<T, R1, INV>(x, tw, R2);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            Y[(q * R1 + k1) * tk + t] = k1 == 0 ? x[k1] : twmul<T, INV>(x[k1], __ldg(tw + q * k1));
    }
    __syncthreads();
    // every thread of the block reaches each barrier below: idle threads skip work, not barriers
    const bool p2 = q < R1;
    C<T> y[R2];
    if (p2) {
#pragma unroll
        for (int j2 = 0; j2 < R2; ++j2) y[j2] = Y[(j2 * R1 + q) * tk + t];
        dft_reg<T, R2, INV>(y, tw, R1);                  // y[k2] = X[q + R1 k2]
        if (!SOLVE && ok) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) a.spec[base + (size_t)(q + R1 * k2) * estride] = y[k2];
        }
    }
    if (!SOLVE) return;
    if (p2) {
        // modal division: -norm/(lx+ly+lz) (zero mode -> 0), or norm/(1 + hcoef lam)
        const T lz = __ldg(tb.lamz + blockIdx.y);
        const T lx = ok ? __ldg(tb.lamx + kx) : T(0);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
            const T lam = lx + __ldg(tb.lamy + q + R1 * k2) + lz;
            const T f = a.hcoef > T(0) ? T(a.norm) / (T(1) + a.hcoef * lam)
                                       : (lam == T(0) ? T(0) : T(-a.norm) / lam);
            y[k2] = mk<T>(y[k2].x * f, y[k2].y * f);
        }
        // inverse: R2-point DFT over k2, twiddle W_n^-(j2 q), exchange, R1-point DFT over k1
        dft_reg<T, R2, true>(y, tw, R1);
    }
    __syncthreads();                                     // every thread has read Y
    if (p2) {
#pragma unroll
        for (int j2 = 0; j2 < R2; ++j2)
            Y[(j2 * R1 + q) * tk + t] = j2 == 0 ? y[j2] : twmul<T, true>(y[j2], __ldg(tw + j2 * q));
    }
    __syncthreads();
    if (q >= R2) return;
    C<T> x[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) x[k1] = Y[(q * R1 + k1) * tk + t];
    dft_reg<T, R1, true>(x, tw, R2);                     // x[j1] = x_(R2 j1 + q)
    if (ok) {
#pragma unroll
        for (int j1 = 0; j1 < R1; ++j1) a.spec[base + (size_t)(R2 * j1 + q) * estride] = x[j1];
    }
}
template <typename T, bool INV, bool SOLVE, int R1, int R2>
__global__ void __launch_bounds__(256)
k_fft_col_r(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a, int axis_y, size_t estride,
            size_t ostride, int tk) {
    k_fft_col_r_body<T, INV, SOLVE, R1, R2>(g, tb, a, axis_y, estride, ostride, tk);
}
template <typename T, bool INV, bool SOLVE, int R1, int R2>
__global__ void __launch_bounds__(256)
k_fft_col_r_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p, int axis_y, size_t estride, size_t ostride, int tk) {
    k_fft_col_r_body<T, INV, SOLVE, R1, R2>(g, tb, p.a[blockIdx.z], axis_y, estride, ostride, tk);
}


// S4 + S5(x) for nx = R1 R2 (powers of two, 16 .. 256), as k_div_fftx with the
// two-pass register-resident FFT: threadIdx.y picks one of the block's complex lines
// (real lines 2L and 2L+1), threadIdx.x = j2 (pass 1), k1 (pass 2), then m (split).
// The exchange buffer of a line is R1 rows of R2+1 (padded against bank conflicts).
template <typename T, int R1, int R2>
__device__ __forceinline__ void k_div_fftx_r_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a) {
    pdl_wait();
    pdl_trigger();
    constexpr int n = R1 * R2, RM = R1 > R2 ? R1 : R2, LW = R1 * (R2 + 1);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int q = threadIdx.x;
    C<T>* Y = reinterpret_cast<C<T>*>(smraw) + (size_t)threadIdx.y * LW;
    const int NL = g.ny * g.nz, nxh = n / 2 + 1;
    const int L0 = 2 * (blockIdx.x * blockDim.y + threadIdx.y), L1 = L0 + 1;
    const bool ok0 = L0 < NL, ok1 = L1 < NL;
    const C<T>* tw = tb.twx;
    if (q < R2) {
        C<T> x[R1];
        if (a.rhs) {
#pragma unroll
            for (int j1 = 0; j1 < R1; ++j1) {
                const int i = R2 * j1 + q;
                x[j1] = mk<T>(ok0 ? __ldg(a.rhs + (size_t)L0 * n + i) : T(0), ok1 ? __ldg(a.rhs + (size_t)L1 * n + i) : T(0));
            }
        } else {
            const DivRows<T> r0 = div_rows(g, a, ok0 ? L0 : 0), r1 = div_rows(g, a, ok1 ? L1 : 0);
            // the second line's v row below is the first line's v row (same plane, the
            // next row): reuse its loads
            const bool share = r1.vm == r0.v;
#pragma unroll
            for (int j1 = 0; j1 < R1; ++j1) {
                const int i = R2 * j1 + q, im = i > 0 ? i - 1 : n - 1;
                const T v0 = __ldg(r0.v + i);
                const T d0 = (__ldg(r0.u + i) - __ldg(r0.u + im)) * g.idx
                             + (v0 - (r0.vm ? __ldg(r0.vm + i) : T(0))) * g.idy
                             + (__ldg(r0.w + i) - __ldg(r0.wm + i)) * g.idz;
                const T vm1 = share ? v0 : (r1.vm ? __ldg(r1.vm + i) : T(0));
                const T d1 = (__ldg(r1.u + i) - __ldg(r1.u + im)) * g.idx + (__ldg(r1.v + i) - vm1) * g.idy
                             + (__ldg(r1.w + i) - __ldg(r1.wm + i)) * g.idz;
                x[j1] = mk<T>(ok0 ? d0 * a.rscale : T(0), ok1 ? d1 * a.rscale : T(0));
            }
        }
        dft_reg<T, R1, false>(x, tw, R2);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            Y[k1 * (R2 + 1) + q] = k1 == 0 ? x[k1] : twmul<T, false>(x[k1], __ldg(tw + q * k1));
    }
    __syncthreads();
    C<T> y[R2];
    if (q < R1) {
#pragma unroll
        for (int j2 = 0; j2 < R2; ++j2) y[j2] = Y[q * (R2 + 1) + j2];
        dft_reg<T, R2, false>(y, tw, R1);                // y[k2] = Z[q + R1 k2]
    }
    __syncthreads();
    if (q < R1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) Y[q + R1 * k2] = y[k2];
    }
    __syncthreads();
    // split the packed pair: A_m = (Z_m + conj Z_{n-m})/2, B_m = (Z_m - conj Z_{n-m})/(2i)
    if (!ok0) return;
    for (int m = q; m < nxh; m += RM) {
        const C<T> Z = Y[m];
        const C<T> Zr = Y[m == 0 ? 0 : n - m];
        a.spec[(size_t)L0 * nxh + m] = mk<T>(T(0.5) * (Z.x + Zr.x), T(0.5) * (Z.y - Zr.y));
        if (ok1) a.spec[(size_t)L1 * nxh + m] = mk<T>(T(0.5) * (Z.y + Zr.y), T(0.5) * (Zr.x - Z.x));
    }
}
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256)
k_div_fftx_r(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a) {
    k_div_fftx_r_body<T, R1, R2>(g, tb, a);
}
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256)
k_div_fftx_r_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p) {
    k_div_fftx_r_body<T, R1, R2>(g, tb, p.a[blockIdx.z]);
}


// S7(x) for nx = R1 R2, as k_ifftx with the two-pass register-resident FFT.
template <typename T, int R1, int R2>
__device__ __forceinline__ void k_ifftx_r_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a) {
    pdl_wait();
    pdl_trigger();
    constexpr int n = R1 * R2, LW = R1 * (R2 + 1), half = n / 2, nxh = n / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int q = threadIdx.x;
    C<T>* Y = reinterpret_cast<C<T>*>(smraw) + (size_t)threadIdx.y * LW;
    const int NL = g.ny * g.nz;
    const int L0 = 2 * (blockIdx.x * blockDim.y + threadIdx.y), L1 = L0 + 1;
    const bool ok0 = L0 < NL, ok1 = L1 < NL;
    const C<T>* tw = tb.twx;
    if (q < R2) {
        C<T> x[R1];
#pragma unroll
        for (int j1 = 0; j1 < R1; ++j1) {
            // packed pair at m: A_m + i B_m with the Hermitian extension of both lines
            const int m = R2 * j1 + q;
            const int mm = m <= half ? m : n - m;
            C<T> A = mk<T>(T(0), T(0)), B = mk<T>(T(0), T(0));
            if (ok0) A = a.spec[(size_t)L0 * nxh + mm];
            if (ok1) B = a.spec[(size_t)L1 * nxh + mm];
            if (mm == 0 || mm == half) {   // DC and Nyquist of a real line are real
                A.y = T(0);
                B.y = T(0);
            }
            if (m > half) {
                A.y = -A.y;
                B.y = -B.y;
            }
            x[j1] = mk<T>(A.x - B.y, A.y + B.x);
        }
        dft_reg<T, R1, true>(x, tw, R2);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
            Y[k1 * (R2 + 1) + q] = k1 == 0 ? x[k1] : twmul<T, true>(x[k1], __ldg(tw + q * k1));
    }
    __syncthreads();
    if (q >= R1 || !ok0) return;
    C<T> y[R2];
#pragma unroll
    for (int j2 = 0; j2 < R2; ++j2) y[j2] = Y[q * (R2 + 1) + j2];
    dft_reg<T, R2, true>(y, tw, R1);                     // y[k2] = z[q + R1 k2]
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
        const size_t i = q + R1 * k2;
        a.psi[(size_t)L0 * n + i] = y[k2].x * a.out_scale;
        if (ok1) a.psi[(size_t)L1 * n + i] = y[k2].y * a.out_scale;
    }
}
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256)
k_ifftx_r(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a) {
    k_ifftx_r_body<T, R1, R2>(g, tb, a);
}
template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256)
k_ifftx_r_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p) {
    k_ifftx_r_body<T, R1, R2>(g, tb, p.a[blockIdx.z]);
}


// ---- double-single arithmetic (Dekker, "A floating-point technique for
// extending the available precision", 1971; Knuth's two-sum): a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48
// significant bits.  Each operation is rounded as written (__fadd_rn, __fmul_rn,
// __fmaf_rn: no contraction or reassociation by the compiler).
struct DS {
    float hi, lo;
};
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker's fast two-sum)
__device__ __forceinline__ DS ds_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// s + e = a + b exactly for any a, b (Knuth's two-sum)
__device__ __forceinline__ DS ds_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return {s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}
// a - b: the high parts exactly, the low parts with one rounding, then
// renormalised; the error is a few units of 2^-48 (|a| + |b|)
__device__ __forceinline__ DS ds_sub(DS a, DS b) {
    DS s = ds_two_sum(a.hi, -b.hi);
    s.lo = __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo));
    return ds_fast_two_sum(s.hi, s.lo);
}
// a b: the rounding error of hi*hi exactly by one fused multiply-add, the cross
// terms added to it, lo*lo dropped; error a few units of 2^-48 |a b|
__device__ __forceinline__ DS ds_mul(DS a, DS b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ds_fast_two_sum(p, e);
}

// S6 with walls, single-precision states: the sweep of k_thomas_body below in
// double-single arithmetic on the FP32 pipes (GB300 runs FP64 at 1/64 of the
// FP32 rate).  The table holds (m_hi, m_lo, c'_hi, c'_lo) per entry
// (thomas_table_ds), the scratch the forward values as (hi, lo) float pairs.  The
// result is hi + lo rounded once to float.  With about 48 bits in every
// operation the sweep's rounding stays some 2^-40 below the FP32 result even for
// the worst-conditioned (lowest) modes of a 512-row wall-normal system.
__device__ __forceinline__ void thomas_ds_body(const Geo<float>& g, const FFTTables<float>& tb,
                                               const PoissonArgs<float>& a) {
    constexpr int TB = 16;
    const int nxh = g.nx / 2 + 1, ny = g.ny, nz = g.nz;
    const int row = 2 * nxh;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= row * nz) return;
    const int kz = gid / row, t = gid - kz * row;             // t = 2*kx + part
    const int kx = t >> 1;
    const int kzh = kz <= nz - kz ? kz : nz - kz;
    const bool pinned = !a.ttab && kx == 0 && kz == 0;                     // Poisson only
    // entries (m_hi, m_lo, c'_hi, c'_lo) (thomas_table_ds)
    const float4* M = reinterpret_cast<const float4*>(a.ttab ? a.ttab : tb.thomas_m) + (size_t)kzh * ny * nxh + kx;
    float* col = reinterpret_cast<float*>(a.spec + (size_t)kz * ny * nxh) + t;
    float2* D = reinterpret_cast<float2*>(a.scratch) + (size_t)kz * ny * (2 * nxh) + t;
    const size_t rs = 2 * (size_t)nxh;
    const size_t ms = (size_t)nxh;
    const double sub = a.ttab ? a.tsub : tb.idy2;                          // the sub-diagonal
    const float sub_hi = (float)sub;
    const DS lo = {sub_hi, (float)(sub - (double)sub_hi)};
    auto m_at = [&](int j) { return __ldg(reinterpret_cast<const float2*>(M + j * ms)); };
    auto c_at = [&](int j) { return __ldg(reinterpret_cast<const float2*>(M + j * ms) + 1); };

    // ---- forward: d'_j = (r_j - sub d'_{j-1}) m_j, d'_0 = r_0 m_0
    DS d = {0.f, 0.f};
    auto fwd = [&](int jj, float r, float2 m) {
        const DS rr = {(pinned && jj == 0) ? 0.f : r, 0.f};
        const DS mv = {m.x, m.y};
        d = ds_mul(jj > 0 ? ds_sub(rr, ds_mul(lo, d)) : rr, mv);
        D[jj * rs] = make_float2(d.hi, d.lo);
    };
    const int nfull = ny / TB * TB;
    float rf[TB];
    float2 mm[TB];
    if (nfull > 0) {
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            rf[u] = col[u * rs];
            mm[u] = m_at(u);
        }
    }
    for (int jb = 0; jb < nfull; jb += TB) {
        float rn[TB];
        float2 mn[TB];
        const bool more = jb + TB < nfull;
        if (more) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                rn[u] = col[(jb + TB + u) * rs];
                mn[u] = m_at(jb + TB + u);
            }
        }
#pragma unroll
        for (int u = 0; u < TB; ++u) fwd(jb + u, rf[u], mm[u]);
        if (more) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                rf[u] = rn[u];
                mm[u] = mn[u];
            }
        }
    }
    for (int jj = nfull; jj < ny; ++jj) fwd(jj, col[jj * rs], m_at(jj));

    // ---- back substitution: psi_{ny-1} = d'_{ny-1}, psi_j = d'_j - c'_j psi_{j+1}
    DS x = d;
    col[(ny - 1) * rs] = __fadd_rn(x.hi, x.lo);
    auto bwd = [&](int jj, float2 dp, float2 c) {
        x = ds_sub(DS{dp.x, dp.y}, ds_mul(DS{c.x, c.y}, x));
        col[jj * rs] = __fadd_rn(x.hi, x.lo);
    };
    const int top = ny - 2;
    const int nrest = (ny - 1) % TB;
    for (int jj = top; jj > top - nrest; --jj) bwd(jj, D[jj * rs], c_at(jj));
    const int jstart = top - nrest;                 // first row of the first full batch (from the top)
    if (jstart >= 0) {
        float2 dd[TB], cc[TB];
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            dd[u] = D[(jstart - u) * rs];
            cc[u] = c_at(jstart - u);
        }
        for (int jt = jstart; jt >= 0; jt -= TB) {
            float2 dn[TB], cn[TB];
            const bool more = jt - TB >= 0;
            if (more) {
#pragma unroll
                for (int u = 0; u < TB; ++u) {
                    dn[u] = D[(jt - TB - u) * rs];
                    cn[u] = c_at(jt - TB - u);
                }
            }
#pragma unroll
            for (int u = 0; u < TB; ++u) bwd(jt - u, dd[u], cc[u]);
            if (more) {
#pragma unroll
                for (int u = 0; u < TB; ++u) {
                    dd[u] = dn[u];
                    cc[u] = cn[u];
                }
            }
        }
    }
}

// S6 with walls: for each (kx, kz) solve
//   psi_{j-1}/dy^2 - (2/dy^2 + lx + lz) psi_j + psi_{j+1}/dy^2 = r_j
// with Neumann rows at j = 0 and ny-1 and the (0, 0) system pinned by psi_0 = 0,
// in FP64.  Real and imaginary parts are independent recurrences with the same
// real coefficients: one thread per (system, part), numbered densely over
// (kz, kx, part) in warp-sized blocks.  m_j = 1/(b_j - a_j c'_{j-1}) and c'_j come
// from a host-built FP64 table; the forward-sweep values d'_j go to an FP64
// scratch in global memory for the back substitution.  Rows are handled in
// batches of TB whose loads are issued one batch ahead, so the recurrence does
// not wait on a memory round trip per row; rows that do not fill a batch are
// done one by one.  The FFT normalisation is applied later, in the inverse x pass.
template <typename T>
__device__ __forceinline__ void thomas_fp64_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a) {
    constexpr int TB = 16;
    const int nxh = g.nx / 2 + 1, ny = g.ny, nz = g.nz;
    const int row = 2 * nxh;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= row * nz) return;
    const int kz = gid / row, t = gid - kz * row;             // t = 2*kx + part
    const int kx = t >> 1;
    const int kzh = kz <= nz - kz ? kz : nz - kz;
    const bool pinned = !a.ttab && kx == 0 && kz == 0;                     // Poisson only
    const double2* M = (a.ttab ? a.ttab : tb.thomas_m) + (size_t)kzh * ny * nxh + kx;   // (m_j, c'_j)
    T* col = reinterpret_cast<T*>(a.spec + (size_t)kz * ny * nxh) + t;    // this part of (kx, kz)
    double* D = a.scratch + (size_t)kz * ny * (2 * nxh) + t;
    const size_t rs = 2 * (size_t)nxh;                                    // row stride in T / double
    const size_t ms = (size_t)nxh;                                        // row stride of the table
    const double idy2 = a.ttab ? a.tsub : tb.idy2;                        // the sub-diagonal

    // ---- forward: d'_j = (r_j - idy2 d'_{j-1}) m_j, d'_0 = r_0 m_0
    const int nfull = ny / TB * TB;
    double d = 0.0;
    T rf[TB];
    double mm[TB];
    if (nfull > 0) {
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            rf[u] = col[u * rs];
            mm[u] = __ldg(&M[u * ms].x);
        }
    }
    for (int jb = 0; jb < nfull; jb += TB) {
        T rn[TB];
        double mn[TB];
        const bool more = jb + TB < nfull;
        if (more) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                rn[u] = col[(jb + TB + u) * rs];
                mn[u] = __ldg(&M[(jb + TB + u) * ms].x);
            }
        }
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            const int jj = jb + u;
            const double r = (pinned && jj == 0) ? 0.0 : widen_f32(rf[u]);
            const double lo = jj > 0 ? idy2 : 0.0;
            d = (r - lo * d) * mm[u];
            D[jj * rs] = d;
        }
        if (more) {
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                rf[u] = rn[u];
                mm[u] = mn[u];
            }
        }
    }
    for (int jj = nfull; jj < ny; ++jj) {
        const double r = (pinned && jj == 0) ? 0.0 : widen_f32(col[jj * rs]);
        const double lo = jj > 0 ? idy2 : 0.0;
        d = (r - lo * d) * __ldg(&M[jj * ms].x);
        D[jj * rs] = d;
    }

    // ---- back substitution: psi_{ny-1} = d'_{ny-1}, psi_j = d'_j - c'_j psi_{j+1}
    double x = d;
    col[(ny - 1) * rs] = narrow_to(x, (T*)nullptr);
    // the top rows that do not fill a batch, then full batches down to row 0
    const int top = ny - 2;
    const int nrest = (ny - 1) % TB;
    for (int jj = top; jj > top - nrest; --jj) {
        x = D[jj * rs] - __ldg(&M[jj * ms].y) * x;
        col[jj * rs] = narrow_to(x, (T*)nullptr);
    }
    const int jstart = top - nrest;                 // first row of the first full batch (from the top)
    if (jstart >= 0) {
        double dd[TB], cc[TB];
#pragma unroll
        for (int u = 0; u < TB; ++u) {
            dd[u] = D[(jstart - u) * rs];
            cc[u] = __ldg(&M[(jstart - u) * ms].y);
        }
        for (int jt = jstart; jt >= 0; jt -= TB) {
            double dn[TB], cn[TB];
            const bool more = jt - TB >= 0;
            if (more) {
#pragma unroll
                for (int u = 0; u < TB; ++u) {
                    dn[u] = D[(jt - TB - u) * rs];
                    cn[u] = __ldg(&M[(jt - TB - u) * ms].y);
                }
            }
#pragma unroll
            for (int u = 0; u < TB; ++u) {
                x = dd[u] - cc[u] * x;
                col[(jt - u) * rs] = narrow_to(x, (T*)nullptr);
            }
            if (more) {
#pragma unroll
                for (int u = 0; u < TB; ++u) {
                    dd[u] = dn[u];
                    cc[u] = cn[u];
                }
            }
        }
    }
}
template <typename T>
__device__ __forceinline__ void k_thomas_body(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a) {
    pdl_wait();
    pdl_trigger();
    if constexpr (sizeof(T) == 4) {
        if (tb.thomas_ds) thomas_ds_body(g, tb, a);
        else thomas_fp64_body<T>(g, tb, a);
    } else {
        thomas_fp64_body<T>(g, tb, a);
    }
}
template <typename T>
__global__ void __launch_bounds__(32)
k_thomas(const Geo<T> g, const FFTTables<T> tb, const PoissonArgs<T> a) {
    k_thomas_body<T>(g, tb, a);
}
template <typename T>
__global__ void __launch_bounds__(32)
k_thomas_b(const Geo<T> g, const FFTTables<T> tb, const __grid_constant__ PoissonBatch<T> p) {
    k_thomas_body<T>(g, tb, p.a[blockIdx.z]);
}


// S8: u^k = u* - c grad psi at the faces, p += psi; non-finite results raise
// EVP_BIT_NONFINITE.  One thread per pair of x-adjacent cells (nx is even): its
// loads (psi at the pair, the next x cell, the +y and +z pairs; u*, v*, w*, p)
// are independent 8- or 16-byte accesses, so each warp keeps them all in flight;
// neighbours' psi come from L1/L2.
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};
template <typename T>
__device__ __forceinline__ void k_correct_body(const Geo<T>& g, const CorrectArgs<T>& a, int k) {
    using V = typename Pair<T>::type;
    pdl_wait();
    pdl_trigger();
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    unsigned bits = 0;
    if (i < g.nx && j < g.ny) {
        const T c = a.coef;
        const size_t plane = (size_t)g.nx * g.ny;
        const size_t o = (size_t)k * plane, cj = (size_t)j * g.nx + i, c0 = o + cj;
        const bool top = g.walls && j == g.ny - 1;
        auto ld = [](const T* p) { return __ldg(reinterpret_cast<const V*>(p)); };
        const V pc = ld(a.psi + c0);
        const T px1 = __ldg(a.psi + o + (size_t)j * g.nx + wrap(i + 2, g.nx));
        const V py = ld(a.psi + o + (size_t)ycen(g, j + 1) * g.nx + i);
        const V pz = ld(a.psi + (size_t)wrap(k + 1, g.nz) * plane + cj);
        const V us = ld(a.Us + c0), vs = ld(a.Vs + c0), ws = ld(a.Ws + c0);
        V Un, Vn, Wn;
        Un.x = us.x - c * ((pc.y - pc.x) * g.idx);
        Un.y = us.y - c * ((px1 - pc.y) * g.idx);
        Vn.x = top ? T(0) : vs.x - c * ((py.x - pc.x) * g.idy);
        Vn.y = top ? T(0) : vs.y - c * ((py.y - pc.y) * g.idy);
        Wn.x = ws.x - c * ((pz.x - pc.x) * g.idz);
        Wn.y = ws.y - c * ((pz.y - pc.y) * g.idz);
        *reinterpret_cast<V*>(a.U + c0) = Un;
        *reinterpret_cast<V*>(a.V + c0) = Vn;
        *reinterpret_cast<V*>(a.W + c0) = Wn;
        if (a.P) {
            V pn = pc;
            if (!a.p_replace) {
                const V pold = *reinterpret_cast<const V*>(a.P + c0);
                pn.x = pold.x + pc.x;
                pn.y = pold.y + pc.y;
            }
            *reinterpret_cast<V*>(a.P + c0) = pn;
        }
        if (!isfinite(Un.x + Vn.x + Wn.x + Un.y + Vn.y + Wn.y)) bits |= EVP_BIT_NONFINITE;
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits) atomicOr(a.status, bits);
}
template <typename T>
__global__ void __launch_bounds__(256)
k_correct(const Geo<T> g, const CorrectArgs<T> a) {
    k_correct_body<T>(g, a, blockIdx.z);
}
// batch: blockIdx.z = member * nz + plane
template <typename T>
__global__ void __launch_bounds__(256)
k_correct_b(const Geo<T> g, const __grid_constant__ CorrectBatch<T> p) {
    const int mb = blockIdx.z / g.nz;
    k_correct_body<T>(g, p.a[mb], blockIdx.z - mb * g.nz);
}


// FP64 max |div u| of a stored staggered velocity: per cell
// (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy + (w_k - w_{k-1})/dz, the FP32 values
// widened exactly by integer operations (widen_f32), periodic in x and z, in y
// periodic or with v = 0 below the first row (walls).  A non-finite divergence
// raises EVP_BIT_NONFINITE and stays out of the maximum, which is kept as the bit
// pattern of a non-negative double (ordered like the unsigned integer); one
// atomic max per block.  A 32 x 8 tile walks a chunk of z planes, carrying w of
// the plane below.
template <typename T>
__device__ __forceinline__ double wide(T x) {
    if constexpr (sizeof(T) == 4) return widen_f32(x);
    else return x;
}
template <typename T>
__global__ void __launch_bounds__(256)
k_div_residual(const Geo<T> g, const T* __restrict__ U, const T* __restrict__ V, const T* __restrict__ W,
               double idx_d, double idy_d, double idz_d, int kz_chunk, unsigned long long* maxdiv, unsigned* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z * kz_chunk, k1 = min(k0 + kz_chunk, g.nz);
    unsigned long long dmax_b = 0ull;
    unsigned bits = 0;
    if (i < g.nx && j < g.ny) {
        const size_t plane = (size_t)g.nx * g.ny;
        const size_t cj = (size_t)j * g.nx + i;
        const int im = wrap(i - 1, g.nx);
        const int jm = j > 0 ? j - 1 : (g.walls ? -1 : g.ny - 1);
        const size_t cxm = (size_t)j * g.nx + im, cym = (size_t)(jm < 0 ? 0 : jm) * g.nx + i;
        double wm = wide(__ldg(W + (size_t)wrap(k0 - 1, g.nz) * plane + cj));
        for (int k = k0; k < k1; ++k) {
            const size_t o = (size_t)k * plane;
            const double w0 = wide(__ldg(W + o + cj));
            const double vm = jm < 0 ? 0.0 : wide(__ldg(V + o + cym));
            const double dv = (wide(__ldg(U + o + cj)) - wide(__ldg(U + o + cxm))) * idx_d
                              + (wide(__ldg(V + o + cj)) - vm) * idy_d + (w0 - wm) * idz_d;
            wm = w0;
            const unsigned long long ab = (unsigned long long)__double_as_longlong(dv) & 0x7fffffffffffffffull;
            // |dv| finite <=> its exponent field is not all ones
            if (ab >= 0x7ff0000000000000ull) bits |= EVP_BIT_NONFINITE;
            else dmax_b = ab > dmax_b ? ab : dmax_b;
        }
    }
    __shared__ unsigned long long red[8];
    __shared__ unsigned rbits[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, dmax_b, o);
        dmax_b = other > dmax_b ? other : dmax_b;
        bits |= __shfl_xor_sync(0xffffffffu, bits, o);
    }
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp] = dmax_b;
        rbits[warp] = bits;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x * blockDim.y) >> 5;
        dmax_b = lane < nw ? red[lane] : 0ull;
        bits = lane < nw ? rbits[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, dmax_b, o);
            dmax_b = other > dmax_b ? other : dmax_b;
            bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        }
        if (lane == 0) {
            if (dmax_b > 0ull) atomicMax(maxdiv, dmax_b);
            if (bits) atomicOr(status, bits);
        }
    }
}

template <typename T>
size_t col_smem(int n, int tk) { return 2 * (size_t)n * tk * sizeof(C<T>); }

template <typename T>
void set_smem(const void* f, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launch of one pass, single or batched.  Single: the state's arguments by value,
// with programmatic dependent launch when asked.  Batched (pb non-null): the same
// kernel's batched form with the members' arguments in parameter space and
// grid.z = members (the single launches use grid.z = 1).
template <typename T>
struct PassLaunch {
    const PoissonArgs<T>* a;
    const PoissonBatch<T>* pb;
    int nb;
    cudaStream_t st;
    bool pdl;
    template <typename KS, typename KB, typename... R>
    cudaError_t go(KS ks, KB kb, dim3 grid, dim3 block, size_t smem, const Geo<T>& g, const FFTTables<T>& tb,
                   R... rest) const {
        if (pb) {
            set_smem<T>((const void*)kb, smem);
            return launch_k(kb, dim3(grid.x, grid.y, nb), block, smem, st, false, g, tb, *pb, rest...);
        }
        set_smem<T>((const void*)ks, smem);
        return launch_k(ks, grid, block, smem, st, pdl, g, tb, *a, rest...);
    }
};

// Column FFT pass of length n along z (axis_y 0) or y (1) over tk consecutive kx
// per block and one block row per grid.y: the register-resident two-pass kernel
// for n = 16 .. 256 (powers of two), else the Stockham kernel.
template <typename T, bool INV, bool SOLVE>
cudaError_t launch_col(const Geo<T>& g, const FFTTables<T>& tb, const PassLaunch<T>& L, int n, int axis_y,
                       size_t estride, size_t ostride, int tk, unsigned rows) {
    const int nxh = g.nx / 2 + 1;
    const dim3 grid((nxh + tk - 1) / tk, rows);
    const size_t smr = (size_t)n * tk * sizeof(C<T>);
#define EVP_COL_R(R1, R2)                                                                                      \
    L.go(k_fft_col_r<T, INV, SOLVE, R1, R2>, k_fft_col_r_b<T, INV, SOLVE, R1, R2>, grid, dim3(tk, R1 > R2 ? R1 : R2), \
         smr, g, tb, axis_y, estride, ostride, tk)
    switch (n) {
        case 16: return EVP_COL_R(4, 4);
        case 32: return EVP_COL_R(4, 8);
        case 64: return EVP_COL_R(8, 8);
        case 128: return EVP_COL_R(8, 16);
        case 256: return EVP_COL_R(16, 16);
        default: break;
    }
#undef EVP_COL_R
    return L.go(k_fft_col<T, INV, SOLVE>, k_fft_col_b<T, INV, SOLVE>, grid, dim3(tk, 256 / tk), col_smem<T>(n, tk), g,
                tb, axis_y, estride, ostride, tk);
}

// The chain of Poisson passes (S4-S7): x pass with the right-hand side, z pass,
// periodic y solve or Thomas sweep, inverse z and inverse x passes.
template <typename T>
cudaError_t poisson_chain(const Geo<T>& g, const FFTTables<T>& tb, const PassLaunch<T>& L, int tk,
                          const TimingHook& th) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxh = nx / 2 + 1;
    const int NL = ny * nz;
    // ---- x pass: np complex lines (2 np real lines) per block
    // np complex lines per block, fewer on small grids so that every SM gets blocks
    const int npairs = (NL + 1) / 2;
    int np = nx >= 2048 ? 1 : 2048 / nx;
    while (np > 1 && (npairs + np - 1) / np < 2 * 152) np /= 2;
    const int tx = nx >= 512 ? 128 : (nx >= 256 ? 64 : 32);
    dim3 bx(tx, 256 / tx);
    dim3 gx((npairs + np - 1) / np);
    const size_t smx = 2 * (size_t)np * nx * sizeof(C<T>);
    // the register-resident x passes for nx = 16 .. 256 (powers of two)
    int xr1 = 0, xr2 = 0;
    switch (nx) {
        case 16: xr1 = 4; xr2 = 4; break;
        case 32: xr1 = 4; xr2 = 8; break;
        case 64: xr1 = 8; xr2 = 8; break;
        case 128: xr1 = 8; xr2 = 16; break;
        case 256: xr1 = 16; xr2 = 16; break;
        default: break;
    }
    const int xrm = xr1 > xr2 ? xr1 : xr2;
    const int xlines = xr1 ? (sizeof(T) == 4 ? 256 : 128) / xrm : 0;          // complex lines per block
    const dim3 bxr(xrm, xlines ? xlines : 1), gxr(xlines ? (npairs + xlines - 1) / xlines : 1);
    const size_t smxr = (size_t)xlines * xr1 * (xr2 + 1) * sizeof(C<T>);
    th.b(K_DIV_FFTX);
    {
        cudaError_t e;
#define EVP_X_R(K, R1, R2) L.go(K<T, R1, R2>, K##_b<T, R1, R2>, gxr, bxr, smxr, g, tb)
        switch (nx) {
            case 16: e = EVP_X_R(k_div_fftx_r, 4, 4); break;
            case 32: e = EVP_X_R(k_div_fftx_r, 4, 8); break;
            case 64: e = EVP_X_R(k_div_fftx_r, 8, 8); break;
            case 128: e = EVP_X_R(k_div_fftx_r, 8, 16); break;
            case 256: e = EVP_X_R(k_div_fftx_r, 16, 16); break;
            default: e = L.go(k_div_fftx<T>, k_div_fftx_b<T>, gx, bx, smx, g, tb, np);
        }
        if (e) return e;
    }
    th.e(K_DIV_FFTX);

    // ---- forward z
    th.b(K_FFT_Z_FWD);
    if (cudaError_t e = launch_col<T, false, false>(g, tb, L, nz, 0, (size_t)ny * nxh, (size_t)nxh, tk, ny))
        return e;
    th.e(K_FFT_Z_FWD);
    if (!g.walls) {
        th.b(K_SOLVE_Y);
        if (cudaError_t e = launch_col<T, false, true>(g, tb, L, ny, 1, (size_t)nxh, (size_t)ny * nxh, tk, nz))
            return e;
        th.e(K_SOLVE_Y);
    } else {
        // warp-sized blocks spread the chains evenly over the SMs
        const int tt = 32;
        const int chains = 2 * nxh * nz;
        dim3 gt((chains + tt - 1) / tt);
        th.b(K_THOMAS);
        if (cudaError_t e = L.go(k_thomas<T>, k_thomas_b<T>, gt, dim3(tt), 0, g, tb)) return e;
        th.e(K_THOMAS);
    }
    // ---- inverse z
    th.b(K_FFT_Z_INV);
    if (cudaError_t e = launch_col<T, true, false>(g, tb, L, nz, 0, (size_t)ny * nxh, (size_t)nxh, tk, ny))
        return e;
    th.e(K_FFT_Z_INV);
    th.b(K_IFFTX);
    {
        cudaError_t e;
        switch (nx) {
            case 16: e = EVP_X_R(k_ifftx_r, 4, 4); break;
            case 32: e = EVP_X_R(k_ifftx_r, 4, 8); break;
            case 64: e = EVP_X_R(k_ifftx_r, 8, 8); break;
            case 128: e = EVP_X_R(k_ifftx_r, 8, 16); break;
            case 256: e = EVP_X_R(k_ifftx_r, 16, 16); break;
            default: e = L.go(k_ifftx<T>, k_ifftx_b<T>, gx, bx, smx, g, tb, np);
        }
#undef EVP_X_R
        if (e) return e;
    }
    th.e(K_IFFTX);
    return cudaGetLastError();
}

}  // namespace

int fft_radices(int n, int* rad) {
    int s = 0;
    while (n % 4 == 0 && n > 2) { rad[s++] = 4; n /= 4; }
    while (n % 3 == 0) { rad[s++] = 3; n /= 3; }
    while (n % 2 == 0) { rad[s++] = 2; n /= 2; }
    return n == 1 ? s : -1;
}

template <typename T>
cudaError_t launch_poisson(const Geo<T>& g, const FFTTables<T>& tb, const PoissonArgs<T>& a, cudaStream_t st,
                           const TimingHook& th) {
    const PassLaunch<T> L{&a, nullptr, 1, st, th.pdl};
    return poisson_chain<T>(g, tb, L, sizeof(T) == 4 ? 16 : 8, th);
}

template <typename T>
cudaError_t launch_poisson_batch(const Geo<T>& g, const FFTTables<T>& tb, const PoissonBatch<T>& p, int n, int tk,
                                 cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n > EVP_BATCH_MAX) return cudaErrorInvalidValue;
    const PassLaunch<T> L{nullptr, &p, n, st, false};
    const TimingHook none{nullptr, nullptr, nullptr};
    return poisson_chain<T>(g, tb, L, tk, none);
}

template <typename T>
cudaError_t launch_correct(const Geo<T>& g, const CorrectArgs<T>& a, cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx / 2 + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_CORRECT);
    const cudaError_t e = launch_k(k_correct<T>, grid, block, 0, st, th.pdl, g, a);
    if (e != cudaSuccess) return e;
    th.e(K_CORRECT);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_div_residual(const Geo<T>& g, const T* U, const T* V, const T* W, double idx, double idy,
                                double idz, unsigned long long* maxdiv, unsigned* status, cudaStream_t st) {
    dim3 block(32, 8, 1);
    const int tiles = ((g.nx + 31) / 32) * ((g.ny + 7) / 8);
    int chunks = (8 * 152 + tiles - 1) / tiles;
    int kz = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + kz - 1) / kz;
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, chunks);
    k_div_residual<T><<<grid, block, 0, st>>>(g, U, V, W, idx, idy, idz, kz, maxdiv, status);
    return cudaGetLastError();
}

template cudaError_t launch_div_residual<float>(const Geo<float>&, const float*, const float*, const float*, double,
                                               double, double, unsigned long long*, unsigned*, cudaStream_t);
template cudaError_t launch_div_residual<double>(const Geo<double>&, const double*, const double*, const double*,
                                                double, double, double, unsigned long long*, unsigned*, cudaStream_t);
template cudaError_t launch_poisson<float>(const Geo<float>&, const FFTTables<float>&, const PoissonArgs<float>&,
                                           cudaStream_t, const TimingHook&);
template cudaError_t launch_poisson<double>(const Geo<double>&, const FFTTables<double>&,
                                            const PoissonArgs<double>&, cudaStream_t, const TimingHook&);
template <typename T>
cudaError_t launch_correct_batch(const Geo<T>& g, const CorrectBatch<T>& p, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dim3 block(32, 8, 1);
    dim3 grid((g.nx / 2 + 31) / 32, (g.ny + 7) / 8, g.nz * n);
    return launch_k(k_correct_b<T>, grid, block, 0, st, false, g, p);
}

template cudaError_t launch_poisson_batch<float>(const Geo<float>&, const FFTTables<float>&,
                                                 const PoissonBatch<float>&, int, int, cudaStream_t);
template cudaError_t launch_poisson_batch<double>(const Geo<double>&, const FFTTables<double>&,
                                                  const PoissonBatch<double>&, int, int, cudaStream_t);
template cudaError_t launch_correct_batch<float>(const Geo<float>&, const CorrectBatch<float>&, int, cudaStream_t);
template cudaError_t launch_correct_batch<double>(const Geo<double>&, const CorrectBatch<double>&, int,
                                                  cudaStream_t);
template cudaError_t launch_correct<float>(const Geo<float>&, const CorrectArgs<float>&, cudaStream_t,
                                           const TimingHook&);
template cudaError_t launch_correct<double>(const Geo<double>&, const CorrectArgs<double>&, cudaStream_t,
                                            const TimingHook&);

}  // namespace evp
