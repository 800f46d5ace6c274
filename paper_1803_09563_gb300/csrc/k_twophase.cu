// S9 + S10: level set, interface force and the AB2 momentum predictor of the
// two-phase step (Secs. 3.2.1 and 3.2.2).
//
//   k_ls_stage      one TVD-RK3 stage of the level-set advection (Eq. ls-adv,
//                   WENO5 upwinded by the centre velocity) or of the
//                   re-distancing equation (Eq. reinit, Godunov |grad phi| from
//                   the WENO5 one-sided derivatives, S(phi0) = phi0/sqrt(phi0^2 + h^2))
//   k_iface_a       H(phi), n = grad phi/|grad phi| (central), per-block sums of 1 - H
//   k_sum_partials  FP64 sum of the block sums (fixed order: deterministic)
//   k_mass_*        mass-preserving uniform shift of phi: block sums of 1 - H and
//                   delta at phi + d, Newton update of d on the device, phi += d
//   k_iface_b       kappa = -div n, the CSF force sigma kappa delta(phi) n (Eq. fLS) and
//                   the mean-free Boussinesq buoyancy, at cell centres
//   k_momentum_ab2  RU = -div(uu) + div[mu_s(H)(grad u + grad u^T)] + div tau(mu_p(H)) + f
//                   and u* = u + dt (w1 RU^n + w0 RU^{n-1})   (Eqs. ru, ab2)
// The level-set and interface kernels take one thread per cell with neighbours
// through the read-only cache; the AB2 momentum kernel marches z-planes of tiles
// staged in shared memory.
#include <cfloat>

#include "evp_internal.cuh"
#include "weno.cuh"

namespace evp {

namespace {

template <typename T>
__device__ __forceinline__ T sqr(T x) { return x * x; }

template <typename T, bool REINIT>
__global__ void __launch_bounds__(256) k_ls_stage(const Geo<T> g, const LsArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c0 = lin(g, i, j, k);
    const T* P = a.phis;
    // the 7-point stencils along x, y, z: wrapped or clamped neighbour indices formed
    // once, as 32-bit offsets (a grid has fewer than 2^31 cells)
    const int row = (k * g.ny + j) * g.nx, col = j * g.nx + i, plane = g.nx * g.ny;
    T p[3][7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        p[0][m] = __ldg(P + (row + wrap(i + m - 3, g.nx)));
        p[1][m] = __ldg(P + ((k * g.ny + ycen(g, j + m - 3)) * g.nx + i));
        p[2][m] = __ldg(P + (wrap(k + m - 3, g.nz) * plane + col));
    }
    const T ih[3] = {g.idx, g.idy, g.idz};
    T rhs;
    if (!REINIT) {
        // -u.grad(phi): upwind WENO5 per direction, velocity at the centre
        const T uc = T(0.5) * (ld_uw(g, a.U, i - 1, j, k) + __ldg(a.U + c0));
        const T vc = T(0.5) * (ld_v(g, a.V, i, j - 1, k) + __ldg(a.V + c0));
        const T wc = T(0.5) * (ld_uw(g, a.W, i, j, k - 1) + __ldg(a.W + c0));
        const T vel[3] = {uc, vc, wc};
        T adv = T(0);
        if constexpr (sizeof(T) == 4) {
            // single precision: the x and y reconstructions in the two lanes of the
            // packed f32x2 WENO5 (each lane picks its upwind side), z on its own
            auto side = [&](int d, int m) { return vel[d] > T(0) ? p[d][m] : p[d][6 - m]; };
            auto xy = [&](int m) { return make_float2(side(0, m), side(1, m)); };
            const float2 sxy = upwind_term2(make_float2(fabs(uc) * ih[0], fabs(vc) * ih[1]), xy(0), xy(1), xy(2),
                                            xy(3), xy(4), xy(5));
            const T sz = fabs(wc) * ih[2];
            const T az = wc > T(0) ? upwind_term(sz, p[2][0], p[2][1], p[2][2], p[2][3], p[2][4], p[2][5])
                                   : upwind_term(sz, p[2][6], p[2][5], p[2][4], p[2][3], p[2][2], p[2][1]);
            adv = (sxy.x + sxy.y) + az;
        } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const T s = fabs(vel[d]) * ih[d];
                if (vel[d] > T(0))
                    adv += upwind_term(s, p[d][0], p[d][1], p[d][2], p[d][3], p[d][4], p[d][5]);
                else
                    adv += upwind_term(s, p[d][6], p[d][5], p[d][4], p[d][3], p[d][2], p[d][1]);
            }
        }
        rhs = -adv;
    } else {
        const T f0 = __ldg(a.phi0 + c0);
        const T sg = f0 / sqrt(f0 * f0 + a.h * a.h);
        T sum = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // left-biased (a) and right-biased (b) derivatives; the mirrored stencil
            // gives the negated right-biased one
            const T dl = upwind_term(ih[d], p[d][0], p[d][1], p[d][2], p[d][3], p[d][4], p[d][5]);
            const T dr = -upwind_term(ih[d], p[d][6], p[d][5], p[d][4], p[d][3], p[d][2], p[d][1]);
            const T pos = fmax(sqr(fmax(dl, T(0))), sqr(fmin(dr, T(0))));
            const T neg = fmax(sqr(fmin(dl, T(0))), sqr(fmax(dr, T(0))));
            sum += sg > T(0) ? pos : neg;
        }
        rhs = -sg * (sqrt(sum) - T(1));
    }
    // plain load: the third stage writes phi in place (each cell by its own thread)
    const T pn = a.pt_a != T(0) ? a.phin[c0] : T(0);
    a.out[c0] = a.pt_a * pn + a.pt_b * (p[0][3] + a.dt * rhs);
}

// H and the unit normal at cell centres; per-block FP64 sum of (1 - H)
template <typename T>
__global__ void __launch_bounds__(256) k_iface_a(const Geo<T> g, const IfaceArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double part = 0.0;
    if (i < g.nx && j < g.ny) {
        const size_t c0 = lin(g, i, j, k);
        const T ph = __ldg(a.phi + c0);
        const T eps = a.eps;
        T H;
        if (ph < -eps) H = T(0);
        else if (ph > eps) H = T(1);
        else H = T(0.5) * (T(1) + ph / eps + sin(T(3.14159265358979323846) * ph / eps) * T(0.31830988618379067154));
        a.H[c0] = H;
        part = 1.0 - double(H);
        const T gx = (ld_c(g, a.phi, i + 1, j, k) - ld_c(g, a.phi, i - 1, j, k)) * (T(0.5) * g.idx);
        const T gy = (ld_c(g, a.phi, i, j + 1, k) - ld_c(g, a.phi, i, j - 1, k)) * (T(0.5) * g.idy);
        const T gz = (ld_c(g, a.phi, i, j, k + 1) - ld_c(g, a.phi, i, j, k - 1)) * (T(0.5) * g.idz);
        T mag = sqrt(gx * gx + gy * gy + gz * gz);
        mag = mag > T(1e-12) ? mag : T(1e-12);
        a.n[0][c0] = gx / mag;
        a.n[1][c0] = gy / mag;
        a.n[2][c0] = gz / mag;
    }
    // fixed-shape block reduction -> one partial per block
    __shared__ double red[256];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    red[t] = part;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) red[t] += red[t + s];
        __syncthreads();
    }
    if (t == 0) a.partials[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_sum_partials(const double* partials, int n, double scale, double* out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 256) s += partials[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

// Soft particles: the solid fraction advected like B, one thread per cell
template <typename T>
__global__ void __launch_bounds__(256) k_phis(const Geo<T> g, const PhisArgs<T> a) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c0 = lin(g, i, j, k);
    // centre velocity: mean of the two faces of the cell
    const T uc = T(0.5) * (__ldg(a.U + c0) + ld_uw(g, a.U, i - 1, j, k));
    const T vc = T(0.5) * (__ldg(a.V + c0) + ld_v(g, a.V, i, j - 1, k));
    const T wc = T(0.5) * (__ldg(a.W + c0) + ld_uw(g, a.W, i, j, k - 1));
    const int sx = uc > T(0) ? 1 : -1, sy = vc > T(0) ? 1 : -1, sz = wc > T(0) ? 1 : -1;
    T p[3][6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        p[0][m] = ld_c(g, a.phi, i + (m - 3) * sx, j, k);
        p[1][m] = ld_c(g, a.phi, i, j + (m - 3) * sy, k);
        p[2][m] = ld_c(g, a.phi, i, j, k + (m - 3) * sz);
    }
    const T adv = upwind_term(fabs(uc) * g.idx, p[0][0], p[0][1], p[0][2], p[0][3], p[0][4], p[0][5])
                  + upwind_term(fabs(vc) * g.idy, p[1][0], p[1][1], p[1][2], p[1][3], p[1][4], p[1][5])
                  + upwind_term(fabs(wc) * g.idz, p[2][0], p[2][1], p[2][2], p[2][3], p[2][4], p[2][5]);
    const T R = -adv;
    T inc = a.dt_zeta * R;
    if (a.read_hist) inc += a.dt_xi * a.hist[c0];
    a.phin[c0] = __ldg(a.phi + c0) + inc;
    if (a.write_hist) a.hist[c0] = R;
}

// Mass correction: per-block FP64 sums of 1 - H(phi + d) and delta(phi + d)
template <typename T>
__global__ void __launch_bounds__(256) k_mass_partials(const Geo<T> g, const MassArgs<T> a, int np) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double v = 0.0, ar = 0.0;
    if (i < g.nx && j < g.ny) {
        const T ph = __ldg(a.phi + lin(g, i, j, k)) + T(*a.d);
        const T eps = a.eps;
        T H, D;
        if (ph < -eps) {
            H = T(0);
            D = T(0);
        } else if (ph > eps) {
            H = T(1);
            D = T(0);
        } else {
            const T x = T(3.14159265358979323846) * ph / eps;
            H = T(0.5) * (T(1) + ph / eps + sin(x) * T(0.31830988618379067154));
            D = T(0.5) / eps * (T(1) + cos(x));
        }
        v = 1.0 - double(H);
        ar = double(D);
    }
    __shared__ double rv[256], ra[256];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    rv[t] = v;
    ra[t] = ar;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            rv[t] += rv[t + w];
            ra[t] += ra[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        a.partials[b] = rv[0];
        a.partials[np + b] = ra[0];
    }
}

// Mass correction: sum the block partials (fixed order) and either record the
// volume (mode 0) or take one Newton step d += (V - v0)/A (mode 1)
__global__ void __launch_bounds__(256) k_mass_newton(const double* partials, int np, double dv, double* v0,
                                                     double* d, int mode) {
    __shared__ double rv[256], ra[256];
    double v = 0.0, ar = 0.0;
    for (int q = threadIdx.x; q < np; q += 256) {
        v += partials[q];
        ar += partials[np + q];
    }
    rv[threadIdx.x] = v;
    ra[threadIdx.x] = ar;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            rv[threadIdx.x] += rv[threadIdx.x + w];
            ra[threadIdx.x] += ra[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double V = rv[0] * dv, A = ra[0] * dv;
        if (mode == 0) *v0 = V;
        else if (A > 0.0) *d += (V - *v0) / A;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mass_shift(T* phi, size_t n, const double* d) {
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) phi[c] += T(*d);
}

// CSF force sigma kappa delta(phi) n plus buoyancy (1 - H - mean(1 - H)) drho_g e_y
template <typename T>
__global__ void __launch_bounds__(256) k_iface_b(const Geo<T> g, const IfaceArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c0 = lin(g, i, j, k);
    const T kap = -((ld_c(g, a.n[0], i + 1, j, k) - ld_c(g, a.n[0], i - 1, j, k)) * (T(0.5) * g.idx)
                    + (ld_c(g, a.n[1], i, j + 1, k) - ld_c(g, a.n[1], i, j - 1, k)) * (T(0.5) * g.idy)
                    + (ld_c(g, a.n[2], i, j, k + 1) - ld_c(g, a.n[2], i, j, k - 1)) * (T(0.5) * g.idz));
    const T ph = __ldg(a.phi + c0);
    const T eps = a.eps;
    const T dl = fabs(ph) > eps ? T(0) : T(0.5) / eps * (T(1) + cos(T(3.14159265358979323846) * ph / eps));
    const T s = a.sigma * kap * dl;
    const T buoy = (T(1) - __ldg(a.H + c0)) * a.drho_g - T(*a.mean_1mH * double(a.drho_g));
    a.f[0][c0] = s * __ldg(a.n[0] + c0);
    a.f[1][c0] = s * __ldg(a.n[1] + c0) + buoy;
    a.f[2][c0] = s * __ldg(a.n[2] + c0);
}

// tau component c at a centre from B^n (b: the six components there) with the
// mixture polymer viscosity mu_p(H) (Table 1 inverted)
template <typename T, int MODEL>
__device__ __forceinline__ T tau_value(const MomAB2Args<T>& a, int c, const T* b, T H) {
    const T gm = (a.mu_p1 * H + a.mu_p2 * (T(1) - H)) * a.inv_lam;
    const bool diag = (c == 0 || c == 3 || c == 5);
    if (MODEL == EVP_FENE_P) {
        const T tr = b[0] + b[3] + b[5];
        const T F = a.L2 / (a.L2 - tr);
        return gm * (F * b[c] - (diag ? a.a_fene : T(0)));
    }
    if (MODEL == EVP_NEO_HOOKEAN) return gm * b[c];
    return gm * (b[c] - (diag ? T(1) : T(0)));
}

// One cell (i, j, k) of the AB2 momentum step.  S gives the staged values around
// the cell at offsets (di, dj, dk) in -1 .. 1: S.u, S.v, S.w (faces), S.H, S.tau(c)
// and S.f(q) (centres); the wraps and wall ghost rules were applied when staging.
template <typename T, int MODEL, typename Src>
__device__ __forceinline__ void momentum_ab2_cell(const Geo<T>& g, const MomAB2Args<T>& a, int i, int j, int k,
                                                  const Src& S) {
    const size_t c0 = lin(g, i, j, k);
    auto u = [&](int di, int dj, int dk) { return S.u(di, dj, dk); };
    auto v = [&](int di, int dj, int dk) { return S.v(di, dj, dk); };
    auto w = [&](int di, int dj, int dk) { return S.w(di, dj, dk); };
    auto mu = [&](int di, int dj, int dk) {
        const T H = S.H(di, dj, dk);
        return a.mu_s1 * H + a.mu_s2 * (T(1) - H);
    };
    // viscosity averaged over the 4 centres (0 or d1) x (0 or d2), shifted by (si, sj, sk)
    auto mue = [&](int si, int sj, int sk, int di, int dj, int dk) {
        int a1i = 0, a1j = 0, a1k = 0, a2i = 0, a2j = 0, a2k = 0;
        if (di) {
            a1i = di;
            if (dj) a2j = dj; else a2k = dk;
        } else {
            a1j = dj;
            a2k = dk;
        }
        return T(0.25) * (mu(si, sj, sk) + mu(si + a2i, sj + a2j, sk + a2k) + mu(si + a1i, sj + a1j, sk + a1k)
                          + mu(si + a1i + a2i, sj + a1j + a2j, sk + a1k + a2k));
    };
    auto tau = [&](int c, int di, int dj, int dk) { return S.tau(c, di, dj, dk); };
    // average of tau_c over (0 or d1) x (0 or d2) around the cell; offsets as in the RK3 kernel
    auto tau_e4 = [&](int c, int di, int dj, int dk) {
        int a1i = 0, a1j = 0, a1k = 0, a2i = 0, a2j = 0, a2k = 0;
        if (di) {
            a1i = di;
            if (dj) a2j = dj; else a2k = dk;
        } else {
            a1j = dj;
            a2k = dk;
        }
        return T(0.25) * (tau(c, 0, 0, 0) + tau(c, a2i, a2j, a2k) + tau(c, a1i, a1j, a1k)
                          + tau(c, a1i + a2i, a1j + a2j, a1k + a2k));
    };
    const T h = T(0.5);
    const T u0 = u(0, 0, 0), v0 = v(0, 0, 0), w0 = w(0, 0, 0);
    const T ix = g.idx, iy = g.idy, iz = g.idz;

    // ---- div(uu) (same discretisation as the RK3 predictor)
    const T Ax = (sqr(h * (u0 + u(1, 0, 0))) - sqr(h * (u(-1, 0, 0) + u0))) * ix
                 + (h * (u0 + u(0, 1, 0)) * h * (v0 + v(1, 0, 0)) - h * (u(0, -1, 0) + u0) * h * (v(0, -1, 0) + v(1, -1, 0))) * iy
                 + (h * (u0 + u(0, 0, 1)) * h * (w0 + w(1, 0, 0)) - h * (u(0, 0, -1) + u0) * h * (w(0, 0, -1) + w(1, 0, -1))) * iz;
    const T Ay = (h * (u0 + u(0, 1, 0)) * h * (v0 + v(1, 0, 0)) - h * (u(-1, 0, 0) + u(-1, 1, 0)) * h * (v(-1, 0, 0) + v0)) * ix
                 + (sqr(h * (v0 + v(0, 1, 0))) - sqr(h * (v(0, -1, 0) + v0))) * iy
                 + (h * (v0 + v(0, 0, 1)) * h * (w0 + w(0, 1, 0)) - h * (v(0, 0, -1) + v0) * h * (w(0, 0, -1) + w(0, 1, -1))) * iz;
    const T Az = (h * (u0 + u(0, 0, 1)) * h * (w0 + w(1, 0, 0)) - h * (u(-1, 0, 0) + u(-1, 0, 1)) * h * (w(-1, 0, 0) + w0)) * ix
                 + (h * (v0 + v(0, 0, 1)) * h * (w0 + w(0, 1, 0)) - h * (v(0, -1, 0) + v(0, -1, 1)) * h * (w(0, -1, 0) + w0)) * iy
                 + (sqr(h * (w0 + w(0, 0, 1))) - sqr(h * (w(0, 0, -1) + w0))) * iz;

    // ---- div[mu (grad u + grad u^T)], normal stresses at centres, shear at edges
    auto sxx = [&](int di) { return T(2) * mu(di, 0, 0) * (u(di, 0, 0) - u(di - 1, 0, 0)) * ix; };
    auto syy = [&](int dj) { return T(2) * mu(0, dj, 0) * (v(0, dj, 0) - v(0, dj - 1, 0)) * iy; };
    auto szz = [&](int dk) { return T(2) * mu(0, 0, dk) * (w(0, 0, dk) - w(0, 0, dk - 1)) * iz; };
    // shear stress at the xy edge (i+si+1/2, j+sj+1/2), etc.
    auto sxy = [&](int si, int sj) {
        return mue(si, sj, 0, 1, 1, 0) * ((u(si, sj + 1, 0) - u(si, sj, 0)) * iy + (v(si + 1, sj, 0) - v(si, sj, 0)) * ix);
    };
    auto sxz = [&](int si, int sk) {
        return mue(si, 0, sk, 1, 0, 1) * ((u(si, 0, sk + 1) - u(si, 0, sk)) * iz + (w(si + 1, 0, sk) - w(si, 0, sk)) * ix);
    };
    auto syz = [&](int sj, int sk) {
        return mue(0, sj, sk, 0, 1, 1) * ((v(0, sj, sk + 1) - v(0, sj, sk)) * iz + (w(0, sj + 1, sk) - w(0, sj, sk)) * iy);
    };
    const T Vx = (sxx(1) - sxx(0)) * ix + (sxy(0, 0) - sxy(0, -1)) * iy + (sxz(0, 0) - sxz(0, -1)) * iz;
    const T Vy = (sxy(0, 0) - sxy(-1, 0)) * ix + (syy(1) - syy(0)) * iy + (syz(0, 0) - syz(0, -1)) * iz;
    const T Vz = (sxz(0, 0) - sxz(-1, 0)) * ix + (syz(0, 0) - syz(-1, 0)) * iy + (szz(1) - szz(0)) * iz;

    // ---- div tau^n with mu_p(H)
    T dtx = T(0), dty = T(0), dtz = T(0);
    if (MODEL != EVP_NEWTONIAN) {
        dtx = (tau(0, 1, 0, 0) - tau(0, 0, 0, 0)) * ix + (tau_e4(1, 1, 1, 0) - tau_e4(1, 1, -1, 0)) * iy
              + (tau_e4(2, 1, 0, 1) - tau_e4(2, 1, 0, -1)) * iz;
        dty = (tau_e4(1, 1, 1, 0) - tau_e4(1, -1, 1, 0)) * ix + (tau(3, 0, 1, 0) - tau(3, 0, 0, 0)) * iy
              + (tau_e4(4, 0, 1, 1) - tau_e4(4, 0, 1, -1)) * iz;
        dtz = (tau_e4(2, 1, 0, 1) - tau_e4(2, -1, 0, 1)) * ix + (tau_e4(4, 0, 1, 1) - tau_e4(4, 0, -1, 1)) * iy
              + (tau(5, 0, 0, 1) - tau(5, 0, 0, 0)) * iz;
    }

    // ---- interface force: mean of the two centres next to each face
    const T Fx = h * (S.f(0, 0, 0, 0) + S.f(0, 1, 0, 0));
    const T Fy = h * (S.f(1, 0, 0, 0) + S.f(1, 0, 1, 0));
    const T Fz = h * (S.f(2, 0, 0, 0) + S.f(2, 0, 0, 1));

    T Nx, Ny, Nz;
    if (a.rho_ratio > T(0)) {
        // density contrast: 1/rho on the stress terms, (1 - rho_bar/rho) g per unit mass
        auto rho = [&](int di, int dj, int dk) {
            const T Hc = S.H(di, dj, dk);
            return Hc + a.rho_ratio * (T(1) - Hc);
        };
        const T r0 = rho(0, 0, 0);
        const T rfx = h * (r0 + rho(1, 0, 0)), rfy = h * (r0 + rho(0, 1, 0)), rfz = h * (r0 + rho(0, 0, 1));
        const double m = *a.mean_1mH;
        const T rbar = T((1.0 - m) + double(a.rho_ratio) * m);
        Nx = -Ax + (Vx + dtx + Fx) / rfx;
        Ny = -Ay + (Vy + dty + Fy) / rfy + (T(1) - rbar / rfy) * (-a.gravity);
        Nz = -Az + (Vz + dtz + Fz) / rfz;
    } else {
        Nx = -Ax + Vx + dtx + Fx;
        Ny = -Ay + Vy + dty + Fy;
        Nz = -Az + Vz + dtz + Fz;
    }
    T ux = a.w1dt * Nx, uy = a.w1dt * Ny, uz = a.w1dt * Nz;
    if (a.read_hist) {
        ux += a.w0dt * a.NH[0][c0];
        uy += a.w0dt * a.NH[1][c0];
        uz += a.w0dt * a.NH[2][c0];
    }
    a.Us[c0] = u0 + ux;
    a.Vs[c0] = (g.walls && j == g.ny - 1) ? T(0) : v0 + uy;
    a.Ws[c0] = w0 + uz;
    a.NH[0][c0] = Nx;
    a.NH[1][c0] = Ny;
    a.NH[2][c0] = Nz;
}

// z-marching tiles of the AB2 momentum step: a 32 x 4 tile walks a chunk of z
// planes.  Planes k-1, k, k+1 of u, v, w, H and tau (built once per staged cell
// from B^n and H, instead of once per stencil use) and planes k, k+1 of the
// interface force sit in shared memory with a one-cell halo in x and y, staged
// with the periodic wraps and the wall ghost rules; the raw values of plane k+2
// are loaded into registers before plane k is computed.
constexpr int AB_TX = 32, AB_TY = 4, AB_NT = AB_TX * AB_TY;
constexpr int AB_W = AB_TX + 2, AB_H = AB_TY + 2, AB_PL = AB_W * AB_H;
constexpr int AB_NE = (AB_PL + AB_NT - 1) / AB_NT;          // staged cells per thread

template <typename T>
struct Ab2Smem {
    T U[3][AB_PL], V[3][AB_PL], W[3][AB_PL], H[3][AB_PL];    // ring slot = plane mod 3
    T TAU[6][3][AB_PL];
    T F[3][2][AB_PL];                                       // slot = plane mod 2
};

template <typename T>
struct Ab2Src {
    const Ab2Smem<T>* sm;
    int o;          // the cell in a plane tile
    int sl[3];      // slots of planes k-1, k, k+1
    int fs[2];      // force slots of planes k, k+1
    __device__ __forceinline__ int at(int di, int dj) const { return o + dj * AB_W + di; }
    __device__ __forceinline__ T u(int di, int dj, int dk) const { return sm->U[sl[1 + dk]][at(di, dj)]; }
    __device__ __forceinline__ T v(int di, int dj, int dk) const { return sm->V[sl[1 + dk]][at(di, dj)]; }
    __device__ __forceinline__ T w(int di, int dj, int dk) const { return sm->W[sl[1 + dk]][at(di, dj)]; }
    __device__ __forceinline__ T H(int di, int dj, int dk) const { return sm->H[sl[1 + dk]][at(di, dj)]; }
    __device__ __forceinline__ T tau(int c, int di, int dj, int dk) const {
        return sm->TAU[c][sl[1 + dk]][at(di, dj)];
    }
    __device__ __forceinline__ T f(int q, int di, int dj, int dk) const { return sm->F[q][fs[dk]][at(di, dj)]; }
};

template <typename T, int MODEL>
__global__ void __launch_bounds__(AB_NT) k_momentum_ab2(const Geo<T> g, const MomAB2Args<T> a, int kz_chunk) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Ab2Smem<T>& sm = *reinterpret_cast<Ab2Smem<T>*>(smraw);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * AB_TX + tx;
    const int i0 = blockIdx.x * AB_TX, j0 = blockIdx.y * AB_TY;
    const int k0 = blockIdx.z * kz_chunk, k1 = min(k0 + kz_chunk, g.nz);
    const int i = i0 + tx, j = j0 + ty;
    const bool active = i < g.nx && j < g.ny;
    constexpr bool STRESS = MODEL != EVP_NEWTONIAN;
    // raw values of one staged plane for this thread's cells
    T ru[AB_NE], rv[AB_NE], rw[AB_NE], rH[AB_NE], rB[6][AB_NE], rf[3][AB_NE];
    auto load = [&](int q) {
#pragma unroll
        for (int r = 0; r < AB_NE; ++r) {
            const int e = tid + r * AB_NT;
            if (e >= AB_PL) continue;
            const int ly = e / AB_W, lx = e - ly * AB_W;
            // the halo of a ragged tile may reach past one period of a short x
            const int gi = ((i0 - 1 + lx) % g.nx + g.nx) % g.nx, gj = j0 - 1 + ly;
            ru[r] = ld_uw(g, a.U, gi, gj, q);
            rv[r] = ld_v(g, a.V, gi, gj, q);
            rw[r] = ld_uw(g, a.W, gi, gj, q);
            rH[r] = ld_c(g, a.H, gi, gj, q);
#pragma unroll
            for (int c = 0; c < 6; ++c) rB[c][r] = STRESS ? ld_c(g, a.B[c], gi, gj, q) : T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) rf[c][r] = ld_c(g, a.f[c], gi, gj, q);
        }
    };
    auto store = [&](int q) {
        const int s3 = (q + 3) % 3, s2 = q & 1;
#pragma unroll
        for (int r = 0; r < AB_NE; ++r) {
            const int e = tid + r * AB_NT;
            if (e >= AB_PL) continue;
            sm.U[s3][e] = ru[r];
            sm.V[s3][e] = rv[r];
            sm.W[s3][e] = rw[r];
            sm.H[s3][e] = rH[r];
            if (STRESS) {
                T b[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) b[c] = rB[c][r];
#pragma unroll
                for (int c = 0; c < 6; ++c) sm.TAU[c][s3][e] = tau_value<T, MODEL>(a, c, b, rH[r]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) sm.F[c][s2][e] = rf[c][r];
        }
    };
    for (int q = k0 - 1; q <= k0 + 1; ++q) {
        load(q);
        store(q);
    }
    __syncthreads();
    Ab2Src<T> src;
    src.sm = &sm;
    src.o = (ty + 1) * AB_W + tx + 1;
    for (int k = k0; k < k1; ++k) {
        const bool more = k + 2 <= k1;
        if (more) load(k + 2);
        src.sl[0] = (k + 2) % 3;
        src.sl[1] = k % 3;
        src.sl[2] = (k + 1) % 3;
        src.fs[0] = k & 1;
        src.fs[1] = (k + 1) & 1;
        if (active) momentum_ab2_cell<T, MODEL>(g, a, i, j, k, src);
        __syncthreads();
        if (more) store(k + 2);
        __syncthreads();
    }
}

// density at a centre from the Heaviside: rho_1 = 1 (H = 1), rho_2 = rho_ratio
template <typename T>
__device__ __forceinline__ T rho_c(const Geo<T>& g, const SplitArgs<T>& a, int i, int j, int k) {
    const T H = ld_c(g, a.H, i, j, k);
    return H + a.rho_ratio * (T(1) - H);
}

// p_hat = 2 p^n - p^{n-1} at a centre
template <typename T>
__device__ __forceinline__ T phat(const Geo<T>& g, const SplitArgs<T>& a, int i, int j, int k) {
    return T(2) * ld_c(g, a.P, i, j, k) - ld_c(g, a.Pold, i, j, k);
}

// r = div[(1 - rho_0/rho_f) grad p_hat] + (rho_0/dt) div u*   (Eq. poisson-LS)
template <typename T>
__global__ void __launch_bounds__(256) k_split_rhs(const Geo<T> g, const SplitArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const size_t c0 = lin(g, i, j, k);
    const T r0 = rho_c(g, a, i, j, k), p0 = phat(g, a, i, j, k);
    // flux (1 - rho_0/rho_f) d p_hat / dn through the +1/2 face of (i, j, k) offset by (di, dj, dk)
    auto fx = [&](int di) {
        const T ra = rho_c(g, a, i + di, j, k), rb = rho_c(g, a, i + di + 1, j, k);
        return (T(1) - a.rho0 / (T(0.5) * (ra + rb))) * (phat(g, a, i + di + 1, j, k) - phat(g, a, i + di, j, k)) * g.idx;
    };
    auto fy = [&](int dj) {
        const int jf = j + dj;
        if (g.walls && (jf < 0 || jf >= g.ny - 1)) return T(0);   // no flux through the walls
        const T ra = rho_c(g, a, i, jf, k), rb = rho_c(g, a, i, jf + 1, k);
        return (T(1) - a.rho0 / (T(0.5) * (ra + rb))) * (phat(g, a, i, jf + 1, k) - phat(g, a, i, jf, k)) * g.idy;
    };
    auto fz = [&](int dk) {
        const T ra = rho_c(g, a, i, j, k + dk), rb = rho_c(g, a, i, j, k + dk + 1);
        return (T(1) - a.rho0 / (T(0.5) * (ra + rb))) * (phat(g, a, i, j, k + dk + 1) - phat(g, a, i, j, k + dk)) * g.idz;
    };
    (void)r0;
    (void)p0;
    const T divf = (fx(0) - fx(-1)) * g.idx + (fy(0) - fy(-1)) * g.idy + (fz(0) - fz(-1)) * g.idz;
    const T du = __ldg(a.Us + c0) - ld_uw(g, a.Us, i - 1, j, k);
    const T dv = __ldg(a.Vs + c0) - ld_v(g, a.Vs, i, j - 1, k);
    const T dw = __ldg(a.Ws + c0) - ld_uw(g, a.Ws, i, j, k - 1);
    a.R[c0] = divf + a.rho0 / a.dt * (du * g.idx + dv * g.idy + dw * g.idz);
}

// u^{n+1} = u* - dt [grad p^{n+1}/rho_0 + (1/rho_f - 1/rho_0) grad p_hat]   (Eq. projection-LS)
template <typename T>
__global__ void __launch_bounds__(256) k_split_correct(const Geo<T> g, const SplitArgs<T> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    unsigned bits = 0;
    if (i < g.nx && j < g.ny) {
        const size_t c0 = lin(g, i, j, k);
        const T ir0 = T(1) / a.rho0;
        // corrected face value of component d at the +1/2 face of (ii, jj, kk)
        auto face = [&](int d, int ii, int jj, int kk) {
            int oi = d == 0, oj = d == 1, ok = d == 2;
            if (d == 1 && g.walls && (jj < 0 || jj >= g.ny - 1)) return T(0);
            const T* S = d == 0 ? a.Us : (d == 1 ? a.Vs : a.Ws);
            const T us = d == 1 ? ld_v(g, S, ii, jj, kk) : ld_uw(g, S, ii, jj, kk);
            const T h = d == 0 ? g.idx : (d == 1 ? g.idy : g.idz);
            const T ra = rho_c(g, a, ii, jj, kk), rb = rho_c(g, a, ii + oi, jj + oj, kk + ok);
            const T rf = T(0.5) * (ra + rb);
            const T gp = (ld_c(g, a.R, ii + oi, jj + oj, kk + ok) - ld_c(g, a.R, ii, jj, kk)) * h;
            const T gh = (phat(g, a, ii + oi, jj + oj, kk + ok) - phat(g, a, ii, jj, kk)) * h;
            return us - a.dt * (gp * ir0 + (T(1) / rf - ir0) * gh);
        };
        const T Un = face(0, i, j, k), Vn = face(1, i, j, k), Wn = face(2, i, j, k);
        a.U[c0] = Un;
        a.V[c0] = Vn;
        a.W[c0] = Wn;
        if (!isfinite(Un + Vn + Wn)) bits |= EVP_BIT_NONFINITE;
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && bits) atomicOr(a.status, bits);
}

}  // namespace

template <typename T>
cudaError_t launch_split_rhs(const Geo<T>& g, const SplitArgs<T>& a, cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_DIV_FFTX);
    k_split_rhs<T><<<grid, block, 0, st>>>(g, a);
    th.e(K_DIV_FFTX);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_split_correct(const Geo<T>& g, const SplitArgs<T>& a, cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_CORRECT);
    k_split_correct<T><<<grid, block, 0, st>>>(g, a);
    th.e(K_CORRECT);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ls_stage(const Geo<T>& g, const LsArgs<T>& a, bool reinit, cudaStream_t st,
                            const TimingHook& th) {
    dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_LEVELSET);
    if (reinit)
        k_ls_stage<T, true><<<grid, block, 0, st>>>(g, a);
    else
        k_ls_stage<T, false><<<grid, block, 0, st>>>(g, a);
    th.e(K_LEVELSET);
    return cudaGetLastError();
}

template <typename T>
size_t iface_partials(const Geo<T>& g) {
    return (size_t)((g.nx + 31) / 32) * ((g.ny + 7) / 8) * g.nz;
}

template <typename T>
cudaError_t launch_interface(const Geo<T>& g, const IfaceArgs<T>& a, cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    const int np = (int)iface_partials(g);
    th.b(K_INTERFACE);
    k_iface_a<T><<<grid, block, 0, st>>>(g, a);
    k_sum_partials<<<1, 256, 0, st>>>(a.partials, np, 1.0 / (double(g.nx) * g.ny * g.nz), a.mean_1mH);
    k_iface_b<T><<<grid, block, 0, st>>>(g, a);
    th.e(K_INTERFACE);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_phis(const Geo<T>& g, const PhisArgs<T>& a, cudaStream_t st, const TimingHook& th) {
    dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    th.b(K_LEVELSET);
    k_phis<T><<<grid, block, 0, st>>>(g, a);
    th.e(K_LEVELSET);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mass_correct(const Geo<T>& g, const MassArgs<T>& a, int mode, int iters, cudaStream_t st,
                                const TimingHook& th) {
    dim3 block(32, 8, 1), grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
    const int np = (int)iface_partials(g);
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    th.b(K_LEVELSET);
    cudaError_t e = cudaMemsetAsync(a.d, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    if (mode == 0) {
        k_mass_partials<T><<<grid, block, 0, st>>>(g, a, np);
        k_mass_newton<<<1, 256, 0, st>>>(a.partials, np, a.dv, a.v0, a.d, 0);
    } else {
        for (int it = 0; it < iters; ++it) {
            k_mass_partials<T><<<grid, block, 0, st>>>(g, a, np);
            k_mass_newton<<<1, 256, 0, st>>>(a.partials, np, a.dv, a.v0, a.d, 1);
        }
        k_mass_shift<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.phi, n, a.d);
    }
    th.e(K_LEVELSET);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_momentum_ab2(const Geo<T>& g, int model, const MomAB2Args<T>& a, cudaStream_t st,
                                const TimingHook& th) {
    // z chunks: about four waves of four CTAs per SM; small grids down to one plane
    const int tiles = ((g.nx + AB_TX - 1) / AB_TX) * ((g.ny + AB_TY - 1) / AB_TY);
    int chunks = (4 * 152 * 4 + tiles - 1) / tiles;
    chunks = chunks > g.nz ? g.nz : chunks;
    const int kz = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + kz - 1) / kz;
    const dim3 block(AB_TX, AB_TY, 1), grid((g.nx + AB_TX - 1) / AB_TX, (g.ny + AB_TY - 1) / AB_TY, chunks);
    const size_t smem = sizeof(Ab2Smem<T>);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, block, smem, st>>>(g, a, kz);
    };
    th.b(K_MOMENTUM);
    switch (model) {
        case EVP_NEWTONIAN: go(k_momentum_ab2<T, EVP_NEWTONIAN>); break;
        case EVP_OLDROYD_B: go(k_momentum_ab2<T, EVP_OLDROYD_B>); break;
        case EVP_FENE_P: go(k_momentum_ab2<T, EVP_FENE_P>); break;
        case EVP_SARAMITO: go(k_momentum_ab2<T, EVP_SARAMITO>); break;
        case EVP_NEO_HOOKEAN: go(k_momentum_ab2<T, EVP_NEO_HOOKEAN>); break;
        default: return cudaErrorInvalidValue;
    }
    th.e(K_MOMENTUM);
    return cudaGetLastError();
}

#define EVP_INST(T)                                                                                           \
    template cudaError_t launch_ls_stage<T>(const Geo<T>&, const LsArgs<T>&, bool, cudaStream_t,              \
                                            const TimingHook&);                                               \
    template size_t iface_partials<T>(const Geo<T>&);                                                         \
    template cudaError_t launch_interface<T>(const Geo<T>&, const IfaceArgs<T>&, cudaStream_t,                \
                                             const TimingHook&);                                              \
    template cudaError_t launch_mass_correct<T>(const Geo<T>&, const MassArgs<T>&, int, int, cudaStream_t,    \
                                                const TimingHook&);                                           \
    template cudaError_t launch_phis<T>(const Geo<T>&, const PhisArgs<T>&, cudaStream_t, const TimingHook&);  \
    template cudaError_t launch_momentum_ab2<T>(const Geo<T>&, int, const MomAB2Args<T>&, cudaStream_t,       \
                                                const TimingHook&);                                           \
    template cudaError_t launch_split_rhs<T>(const Geo<T>&, const SplitArgs<T>&, cudaStream_t, const TimingHook&); \
    template cudaError_t launch_split_correct<T>(const Geo<T>&, const SplitArgs<T>&, cudaStream_t,            \
                                                 const TimingHook&);
EVP_INST(float)
EVP_INST(double)
#undef EVP_INST

}  // namespace evp
