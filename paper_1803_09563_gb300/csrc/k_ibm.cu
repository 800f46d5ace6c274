// Discrete-forcing immersed boundary method for rigid particles (Sec. 3.3.2,
// Eqs. IBM a-d and CoVe2), one multi-direct iteration per launch pair:
//   k_ibm_interp   one thread per Lagrangian point: U*_l from the 27 nodes of each
//                  velocity component's lattice (three-point Roma kernel), the
//                  increment dF_l = (U_p + omega_p x r_l - U*_l)/dt_s, accumulated
//   k_ibm_spread   one thread per (point, component): u** += dt_s dF_l delta dV_l
//                  over the 27 nodes (atomic adds: points share nodes)
//   k_ibm_finish   one block per particle: force and torque the fluid exerts on
//                  the particle, -sum F_l dV_l and -sum r_l x F_l dV_l, in FP64
//   k_ibm_integrals  one block per (particle, component): inner-fluid integrals
//                  int u dV and int r x u dV over the nodes of the particle's box,
//                  phi_s from 4^3 sub-samples of each node's control volume
//   k_ibm_update   one thread per particle: Newton-Euler step of a free sphere
//                  (or the prescribed motion), centre by the trapezoidal rule
// Positions and kernel weights are formed in FP64, the fields in their precision.
#include "evp_internal.cuh"

namespace evp {

namespace {

// three-point kernel of Roma et al., r in cells
__device__ __forceinline__ double roma(double r) {
    r = fabs(r);
    if (r <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) * (1.0 / 3.0);
    if (r <= 1.5) {
        const double q = 1.0 - r;
        return (5.0 - 3.0 * r - sqrt(fmax(0.0, 1.0 - 3.0 * q * q))) * (1.0 / 6.0);
    }
    return 0.0;
}

// the three nodes and weights around X along one direction of a lattice whose
// node i sits at x0 + i h (periodic index wrap)
__device__ __forceinline__ void stencil1(double X, double x0, double h, int n, int idx[3], double w[3]) {
    const int base = (int)floor((X - x0) / h + 0.5);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int ii = base - 1 + m;
        w[m] = roma((x0 + ii * h - X) / h);
        int r = ii % n;
        idx[m] = r < 0 ? r + n : r;
    }
}

template <typename T>
__device__ __forceinline__ void stencil3(const IbmArgs<T>& a, int c, const double X[3], int ix[3], int iy[3],
                                         int iz[3], double wx[3], double wy[3], double wz[3]) {
    // component c's lattice: faces (i + 1) h along its own direction, centres (i + 1/2) h otherwise
    const double hx = a.dx, hy = a.dy, hz = a.dz;
    stencil1(X[0], (c == 0 ? 1.0 : 0.5) * hx, hx, a.nx, ix, wx);
    stencil1(X[1], a.y0 + (c == 1 ? 1.0 : 0.5) * hy, hy, a.ny, iy, wy);
    stencil1(X[2], (c == 2 ? 1.0 : 0.5) * hz, hz, a.nz, iz, wz);
}

template <typename T>
__global__ void __launch_bounds__(128) k_ibm_interp(const IbmArgs<T> a, int first) {
    pdl_wait();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.nl) return;
    const int p = a.owner[l];
    const double r[3] = {a.off[3 * l], a.off[3 * l + 1], a.off[3 * l + 2]};
    const double X[3] = {a.centre[3 * p] + r[0], a.centre[3 * p + 1] + r[1], a.centre[3 * p + 2] + r[2]};
    const double* w = a.pomg + 3 * p;
    const double* v = a.pvel + 3 * p;
    // surface velocity U_p + omega_p x r
    const double tgt[3] = {v[0] + w[1] * r[2] - w[2] * r[1], v[1] + w[2] * r[0] - w[0] * r[2],
                           v[2] + w[0] * r[1] - w[1] * r[0]};
    const size_t nxy = (size_t)a.nx * a.ny;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        int ix[3], iy[3], iz[3];
        double wx[3], wy[3], wz[3];
        stencil3(a, c, X, ix, iy, iz, wx, wy, wz);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    s += double(__ldg(a.U[c] + (size_t)iz[k] * nxy + (size_t)iy[j] * a.nx + ix[i])) * wx[i] * wy[j] *
                         wz[k];
        const double dF = (tgt[c] - s) / a.dts;
        a.dF[3 * l + c] = dF;
        a.Facc[3 * l + c] = first ? dF : a.Facc[3 * l + c] + dF;
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_ibm_spread(const IbmArgs<T> a) {
    pdl_wait();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * a.nl) return;
    const int l = t / 3, c = t - 3 * l;
    const int p = a.owner[l];
    const double X[3] = {a.centre[3 * p] + a.off[3 * l], a.centre[3 * p + 1] + a.off[3 * l + 1],
                         a.centre[3 * p + 2] + a.off[3 * l + 2]};
    int ix[3], iy[3], iz[3];
    double wx[3], wy[3], wz[3];
    stencil3(a, c, X, ix, iy, iz, wx, wy, wz);
    // delta dV_l = phi phi phi dV_l / cell; u** += dt_s dF delta dV_l
    const double amp = a.dts * a.dF[3 * l + c] * a.dvl[p] / (a.dx * a.dy * a.dz);
    const size_t nxy = (size_t)a.nx * a.ny;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i)
                atomicAdd(a.U[c] + (size_t)iz[k] * nxy + (size_t)iy[j] * a.nx + ix[i], T(amp * wx[i] * wy[j] * wz[k]));
}

__global__ void __launch_bounds__(128) k_ibm_finish(const double* off, const int* start, const double* dvl,
                                                    const double* Facc, const double* pvel, double* centre,
                                                    double* pforce, double dts) {
    pdl_wait();
    const int p = blockIdx.x;
    __shared__ double red[6][128];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int l = start[p] + threadIdx.x; l < start[p + 1]; l += blockDim.x) {
        const double* F = Facc + 3 * l;
        const double* r = off + 3 * l;
        acc[0] += F[0];
        acc[1] += F[1];
        acc[2] += F[2];
        acc[3] += r[1] * F[2] - r[2] * F[1];
        acc[4] += r[2] * F[0] - r[0] * F[2];
        acc[5] += r[0] * F[1] - r[1] * F[0];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) pforce[6 * p + q] = -red[q][0] * dvl[p];
    }
}

// inner-fluid integrals of particle blockIdx.x from component blockIdx.y of (u, v, w)
template <typename T>
__global__ void __launch_bounds__(256) k_ibm_integrals(const IbmArgs<T> a, const T* u, const T* v, const T* w,
                                                       double* I) {
    pdl_wait();
    const int p = blockIdx.x, c = blockIdx.y;
    const T* F = c == 0 ? u : (c == 1 ? v : w);
    const double R = a.prad[p];
    const double cx = a.centre[3 * p], cy = a.centre[3 * p + 1], cz = a.centre[3 * p + 2];
    // component c's lattice origins (faces along its own axis)
    const double x0 = (c == 0 ? 1.0 : 0.5) * a.dx, y0 = a.y0 + (c == 1 ? 1.0 : 0.5) * a.dy,
                 z0 = (c == 2 ? 1.0 : 0.5) * a.dz;
    // unwrapped node ranges covering [centre - R - h, centre + R + h]
    const int ilo = (int)floor((cx - R - x0) / a.dx) - 1, ihi = (int)ceil((cx + R - x0) / a.dx) + 1;
    int jlo = (int)floor((cy - R - y0) / a.dy) - 1, jhi = (int)ceil((cy + R - y0) / a.dy) + 1;
    const int klo = (int)floor((cz - R - z0) / a.dz) - 1, khi = (int)ceil((cz + R - z0) / a.dz) + 1;
    if (a.walls) {
        jlo = max(jlo, 0);
        jhi = min(jhi, a.ny - 1);
    }
    const int ni = ihi - ilo + 1, nj = jhi - jlo + 1, nk = khi - klo + 1;
    const double cell = a.dx * a.dy * a.dz, R2 = R * R;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const long total = (long)ni * nj * nk;
    for (long q = threadIdx.x; q < total; q += blockDim.x) {
        const int ii = ilo + (int)(q % ni), jj = jlo + (int)((q / ni) % nj), kk = klo + (int)(q / ((long)ni * nj));
        const double rx = x0 + ii * a.dx - cx, ry = y0 + jj * a.dy - cy, rz = z0 + kk * a.dz - cz;
        int inside = 0;
#pragma unroll
        for (int sx = 0; sx < 4; ++sx)
#pragma unroll
            for (int sy = 0; sy < 4; ++sy)
#pragma unroll
                for (int sz = 0; sz < 4; ++sz) {
                    const double px = rx + ((sx + 0.5) * 0.25 - 0.5) * a.dx;
                    const double py = ry + ((sy + 0.5) * 0.25 - 0.5) * a.dy;
                    const double pz = rz + ((sz + 0.5) * 0.25 - 0.5) * a.dz;
                    inside += px * px + py * py + pz * pz < R2;
                }
        if (!inside) continue;
        const int gi = ((ii % a.nx) + a.nx) % a.nx, gj = ((jj % a.ny) + a.ny) % a.ny, gk = ((kk % a.nz) + a.nz) % a.nz;
        const double val = double(__ldg(F + ((size_t)gk * a.ny + gj) * a.nx + gi)) * (inside * (1.0 / 64.0)) * cell;
        const double r[3] = {rx, ry, rz};
        acc[c] += val;
        // (r x u)_a gains r_b u_c and (r x u)_b loses r_a u_c, (c, a, b) cyclic
        const int ca = (c + 1) % 3, cb = (c + 2) % 3;
        acc[3 + ca] += r[cb] * val;
        acc[3 + cb] -= r[ca] * val;
    }
    __shared__ double red[6][256];
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 6) atomicAdd(I + 6 * p + threadIdx.x, red[threadIdx.x][0]);
}

// Newton-Euler step of a free sphere (rho_p/rho_f > 0) or the prescribed motion
template <typename T>
__global__ void k_ibm_update(const IbmArgs<T> a) {
    pdl_wait();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    double* u = a.pvel_w + 3 * p;
    double* w = a.pomg_w + 3 * p;
    double* c = a.centre + 3 * p;
    const double rho = a.pdens[p];
    if (rho > 0.0) {
        const double R = a.prad[p];
        const double vp = 4.0 / 3.0 * 3.14159265358979323846 * R * R * R;
        const double ip = 0.4 * rho * vp * R * R;
        const double* f = a.pforce + 6 * p;
        const double* i0 = a.I0 + 6 * p;
        const double* i1 = a.I1 + 6 * p;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double gd = d == 1 ? -a.gravity : 0.0;
            const double un = u[d] + (a.dts * f[d] + (i1[d] - i0[d]) + a.dts * (rho - 1.0) * vp * gd) / (rho * vp);
            w[d] += (a.dts * f[3 + d] + (i1[3 + d] - i0[3 + d])) / ip;
            c[d] += 0.5 * a.dts * (un + u[d]);
            u[d] = un;
        }
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) c[d] += a.dts * u[d];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_ibm(const IbmArgs<T>& a, const T* const uold[3], int iters, cudaStream_t st,
                       const TimingHook& th) {
    if (a.nl == 0) return cudaSuccess;
    th.b(K_IBM);
    cudaError_t e;
    if (a.any_free) {
        if ((e = cudaMemsetAsync(a.I0, 0, 12 * (size_t)a.np * sizeof(double), st)) != cudaSuccess) return e;
        k_ibm_integrals<T><<<dim3(a.np, 3), 256, 0, st>>>(a, uold[0], uold[1], uold[2], a.I0);
    }
    for (int it = 0; it < iters; ++it) {
        k_ibm_interp<T><<<(a.nl + 127) / 128, 128, 0, st>>>(a, it == 0 ? 1 : 0);
        k_ibm_spread<T><<<(3 * a.nl + 127) / 128, 128, 0, st>>>(a);
    }
    k_ibm_finish<<<a.np, 128, 0, st>>>(a.off, a.start, a.dvl, a.Facc, a.pvel, a.centre, a.pforce, a.dts);
    if (a.any_free) k_ibm_integrals<T><<<dim3(a.np, 3), 256, 0, st>>>(a, a.U[0], a.U[1], a.U[2], a.I1);
    k_ibm_update<T><<<(a.np + 127) / 128, 128, 0, st>>>(a);
    th.e(K_IBM);
    return cudaGetLastError();
}

template cudaError_t launch_ibm<float>(const IbmArgs<float>&, const float* const[3], int, cudaStream_t,
                                       const TimingHook&);
template cudaError_t launch_ibm<double>(const IbmArgs<double>&, const double* const[3], int, cudaStream_t,
                                        const TimingHook&);

}  // namespace evp
