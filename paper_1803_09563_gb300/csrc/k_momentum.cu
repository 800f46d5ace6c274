// S3: momentum predictor of Eqs. NS-num1 and rk3 on the staggered grid.
//
// u* = u^{k-1} + dt [zeta^k N^{k-1} + xi^k N^{k-2} - 2 alpha^k grad p^{k-1}
//                    + alpha^k (div tau^k + div tau^{k-1})]
// N  = -div(uu) + mu_s lap(u) + f
//
// div(uu) by second-order central differences (products at centres and edges),
// the viscous term explicit with the advective weights, div(tau) at faces from
// centre tau with 4-point edge averages for the off-diagonal parts.  One thread
// computes the three faces (i+1/2, j, k), (i, j+1/2, k), (i, j, k+1/2) of cell
// (i, j, k); with walls the top y-face stays zero.
#include "evp_internal.cuh"

namespace evp {

namespace {

template <typename T>
__device__ __forceinline__ T sq(T x) { return x * x; }

// tau component c (xx xy xz yy yz zz) at a centre, from B (Table 1 inverted)
template <typename T, int MODEL>
__device__ __forceinline__ T tau_at(const Geo<T>& g, const ModelConst& mc, const T* const* B,
                                    int c, int i, int j, int k) {
    const T gm = T(mc.gmod);
    const size_t o = lin(g, wrap(i, g.nx), ycen(g, j), wrap(k, g.nz));
    const T bc = __ldg(B[c] + o);
    const bool diag = (c == 0 || c == 3 || c == 5);
    if (MODEL == EVP_FENE_P) {
        const T tr = __ldg(B[0] + o) + __ldg(B[3] + o) + __ldg(B[5] + o);
        const T F = T(mc.L2) / (T(mc.L2) - tr);
        return gm * (F * bc - (diag ? T(mc.a_fene) : T(0)));
    }
    return gm * (bc - (diag ? T(1) : T(0)));
}

// 4-point average of tau_c over the centres (i + {0, di}, j + {0, dj}, k + {0, dk})
// where exactly two of di, dj, dk are non-zero.
template <typename T, int MODEL>
__device__ __forceinline__ T tau_edge(const Geo<T>& g, const ModelConst& mc, const T* const* B, int c,
                                      int i, int j, int k, int di, int dj, int dk) {
    // the two offsets as (o1, o2); summed in the order (0,0), (0,o2), (o1,0), (o1,o2)
    int a1i = 0, a1j = 0, a1k = 0, a2i = 0, a2j = 0, a2k = 0;
    if (di) {
        a1i = di;
        if (dj) a2j = dj; else a2k = dk;
    } else {
        a1j = dj;
        a2k = dk;
    }
    T s = tau_at<T, MODEL>(g, mc, B, c, i, j, k);
    s += tau_at<T, MODEL>(g, mc, B, c, i + a2i, j + a2j, k + a2k);
    s += tau_at<T, MODEL>(g, mc, B, c, i + a1i, j + a1j, k + a1k);
    s += tau_at<T, MODEL>(g, mc, B, c, i + a1i + a2i, j + a1j + a2j, k + a1k + a2k);
    return T(0.25) * s;
}

// div tau at the three faces of cell (i, j, k)
template <typename T, int MODEL>
__device__ __forceinline__ void div_tau(const Geo<T>& g, const ModelConst& mc, const T* const* B,
                                        int i, int j, int k, T& fx, T& fy, T& fz) {
    // x-face (i+1/2, j, k)
    fx = (tau_at<T, MODEL>(g, mc, B, 0, i + 1, j, k) - tau_at<T, MODEL>(g, mc, B, 0, i, j, k)) * g.idx
         + (tau_edge<T, MODEL>(g, mc, B, 1, i, j, k, 1, 1, 0) - tau_edge<T, MODEL>(g, mc, B, 1, i, j, k, 1, -1, 0)) * g.idy
         + (tau_edge<T, MODEL>(g, mc, B, 2, i, j, k, 1, 0, 1) - tau_edge<T, MODEL>(g, mc, B, 2, i, j, k, 1, 0, -1)) * g.idz;
    // y-face (i, j+1/2, k)
    fy = (tau_edge<T, MODEL>(g, mc, B, 1, i, j, k, 1, 1, 0) - tau_edge<T, MODEL>(g, mc, B, 1, i, j, k, -1, 1, 0)) * g.idx
         + (tau_at<T, MODEL>(g, mc, B, 3, i, j + 1, k) - tau_at<T, MODEL>(g, mc, B, 3, i, j, k)) * g.idy
         + (tau_edge<T, MODEL>(g, mc, B, 4, i, j, k, 0, 1, 1) - tau_edge<T, MODEL>(g, mc, B, 4, i, j, k, 0, 1, -1)) * g.idz;
    // z-face (i, j, k+1/2)
    fz = (tau_edge<T, MODEL>(g, mc, B, 2, i, j, k, 1, 0, 1) - tau_edge<T, MODEL>(g, mc, B, 2, i, j, k, -1, 0, 1)) * g.idx
         + (tau_edge<T, MODEL>(g, mc, B, 4, i, j, k, 0, 1, 1) - tau_edge<T, MODEL>(g, mc, B, 4, i, j, k, 0, -1, 1)) * g.idy
         + (tau_at<T, MODEL>(g, mc, B, 5, i, j, k + 1) - tau_at<T, MODEL>(g, mc, B, 5, i, j, k)) * g.idz;
}

template <typename T, int MODEL>
__global__ void __launch_bounds__(256)
k_momentum(const Geo<T> g, const ModelConst mc, const MomentumArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c0 = lin(g, i, j, k);
    const T* U = a.U;
    const T* V = a.V;
    const T* W = a.W;
    auto u = [&](int di, int dj, int dk) { return ld_uw(g, U, i + di, j + dj, k + dk); };
    auto v = [&](int di, int dj, int dk) { return ld_v(g, V, i + di, j + dj, k + dk); };
    auto w = [&](int di, int dj, int dk) { return ld_uw(g, W, i + di, j + dj, k + dk); };
    const T h = T(0.5);
    const T u0 = u(0, 0, 0), v0 = v(0, 0, 0), w0 = w(0, 0, 0);

    // ---- div(uu) at the three faces
    const T Ax = (sq(h * (u0 + u(1, 0, 0))) - sq(h * (u(-1, 0, 0) + u0))) * g.idx
                 + (h * (u0 + u(0, 1, 0)) * h * (v0 + v(1, 0, 0))
                    - h * (u(0, -1, 0) + u0) * h * (v(0, -1, 0) + v(1, -1, 0))) * g.idy
                 + (h * (u0 + u(0, 0, 1)) * h * (w0 + w(1, 0, 0))
                    - h * (u(0, 0, -1) + u0) * h * (w(0, 0, -1) + w(1, 0, -1))) * g.idz;
    const T Ay = (h * (u0 + u(0, 1, 0)) * h * (v0 + v(1, 0, 0))
                  - h * (u(-1, 0, 0) + u(-1, 1, 0)) * h * (v(-1, 0, 0) + v0)) * g.idx
                 + (sq(h * (v0 + v(0, 1, 0))) - sq(h * (v(0, -1, 0) + v0))) * g.idy
                 + (h * (v0 + v(0, 0, 1)) * h * (w0 + w(0, 1, 0))
                    - h * (v(0, 0, -1) + v0) * h * (w(0, 0, -1) + w(0, 1, -1))) * g.idz;
    const T Az = (h * (u0 + u(0, 0, 1)) * h * (w0 + w(1, 0, 0))
                  - h * (u(-1, 0, 0) + u(-1, 0, 1)) * h * (w(-1, 0, 0) + w0)) * g.idx
                 + (h * (v0 + v(0, 0, 1)) * h * (w0 + w(0, 1, 0))
                    - h * (v(0, -1, 0) + v(0, -1, 1)) * h * (w(0, -1, 0) + w0)) * g.idy
                 + (sq(h * (w0 + w(0, 0, 1))) - sq(h * (w(0, 0, -1) + w0))) * g.idz;

    // ---- mu_s lap(u)
    const T idx2 = g.idx * g.idx, idy2 = g.idy * g.idy, idz2 = g.idz * g.idz;
    const T mu = T(mc.mu_s);
    const T Lu = (u(1, 0, 0) - T(2) * u0 + u(-1, 0, 0)) * idx2 + (u(0, 1, 0) - T(2) * u0 + u(0, -1, 0)) * idy2
                 + (u(0, 0, 1) - T(2) * u0 + u(0, 0, -1)) * idz2;
    const T Lv = (v(1, 0, 0) - T(2) * v0 + v(-1, 0, 0)) * idx2 + (v(0, 1, 0) - T(2) * v0 + v(0, -1, 0)) * idy2
                 + (v(0, 0, 1) - T(2) * v0 + v(0, 0, -1)) * idz2;
    const T Lw = (w(1, 0, 0) - T(2) * w0 + w(-1, 0, 0)) * idx2 + (w(0, 1, 0) - T(2) * w0 + w(0, -1, 0)) * idy2
                 + (w(0, 0, 1) - T(2) * w0 + w(0, 0, -1)) * idz2;

    // ---- body force: uniform dp/dx plus ABC forcing (separable tables)
    T fx = a.dpdx, fy = T(0), fz = T(0);
    if (a.trig) {
        const T* sx = a.trig;
        const T* cx = sx + g.nx;
        const T* sy = cx + g.nx;
        const T* cy = sy + g.ny;
        const T* sz = cy + g.ny;
        const T* cz = sz + g.nz;
        fx += a.abc_amp * (sz[k] + cy[j]);
        fy = a.abc_amp * (sx[i] + cz[k]);
        fz = a.abc_amp * (sy[j] + cx[i]);
    }
    const T Nx = -Ax + mu * Lu + fx;
    const T Ny = -Ay + mu * Lv + fy;
    const T Nz = -Az + mu * Lw + fz;

    // ---- pressure gradient at the faces
    const T p0 = __ldg(a.P + c0);
    const T gpx = (ld_c(g, a.P, i + 1, j, k) - p0) * g.idx;
    const T gpy = (ld_c(g, a.P, i, j + 1, k) - p0) * g.idy;
    const T gpz = (ld_c(g, a.P, i, j, k + 1) - p0) * g.idz;

    T ix = a.zeta * Nx, iy = a.zeta * Ny, iz = a.zeta * Nz;
    if (a.read_hist) {
        ix += a.xi * a.NH[0][c0];
        iy += a.xi * a.NH[1][c0];
        iz += a.xi * a.NH[2][c0];
    }
    const T two_a = T(2) * a.alpha;
    ix -= two_a * gpx;
    iy -= two_a * gpy;
    iz -= two_a * gpz;
    if (MODEL != EVP_NEWTONIAN) {
        T ox, oy, oz, nx_, ny_, nz_;
        div_tau<T, MODEL>(g, mc, a.Bn, i, j, k, nx_, ny_, nz_);
        div_tau<T, MODEL>(g, mc, a.Bo, i, j, k, ox, oy, oz);
        ix += a.alpha * (nx_ + ox);
        iy += a.alpha * (ny_ + oy);
        iz += a.alpha * (nz_ + oz);
    }
    a.Us[c0] = u0 + a.dt * ix;
    a.Vs[c0] = (g.walls && j == g.ny - 1) ? T(0) : v0 + a.dt * iy;
    a.Ws[c0] = w0 + a.dt * iz;
    if (a.write_hist) {
        a.NH[0][c0] = Nx;
        a.NH[1][c0] = Ny;
        a.NH[2][c0] = Nz;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_momentum(const Geo<T>& g, const ModelConst& mc, const MomentumArgs<T>& a,
                            cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_MOMENTUM);
    switch (mc.model) {
        case EVP_NEWTONIAN: k_momentum<T, EVP_NEWTONIAN><<<grid, block, 0, st>>>(g, mc, a); break;
        case EVP_OLDROYD_B: k_momentum<T, EVP_OLDROYD_B><<<grid, block, 0, st>>>(g, mc, a); break;
        case EVP_FENE_P: k_momentum<T, EVP_FENE_P><<<grid, block, 0, st>>>(g, mc, a); break;
        case EVP_SARAMITO: k_momentum<T, EVP_SARAMITO><<<grid, block, 0, st>>>(g, mc, a); break;
        default: return cudaErrorInvalidValue;
    }
    th.e(K_MOMENTUM);
    return cudaGetLastError();
}

template cudaError_t launch_momentum<float>(const Geo<float>&, const ModelConst&, const MomentumArgs<float>&,
                                            cudaStream_t, const TimingHook&);
template cudaError_t launch_momentum<double>(const Geo<double>&, const ModelConst&, const MomentumArgs<double>&,
                                             cudaStream_t, const TimingHook&);

}  // namespace evp
