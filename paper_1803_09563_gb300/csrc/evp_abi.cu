// Host side of libevp: the C ABI of evp.h, the device arena, the constant tables
// (FFT twiddles, modal eigenvalues, Thomas pivots, forcing tables) and the RK3
// orchestration of Sec. 3.3.1 (Eqs. RK-rt, NS-num1, rk3tau, rk3, NS-num2, NS-num3, RK).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "evp_internal.cuh"
#include "evp_state.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace evp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return EVP_ERR_CUDA;
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)


const char* KERNEL_NAMES[K_COUNT] = {"stress_weno_update", "momentum_predictor", "div_fft_x",
                                     "fft_z_forward",      "fft_y_modal_solve",  "thomas_y",
                                     "fft_z_inverse",      "ifft_x_psi",         "project_correct",
                                     "levelset_stage",     "interface_force",    "ibm_forcing"};

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace evp {
// lets other translation units of the library report through evp_last_error()
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace evp


namespace {

cudaEvent_t get_event(evp_state* s) {
    if (!s->ev_free.empty()) {
        cudaEvent_t e = s->ev_free.back();
        s->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void flush_timing(evp_state* s) {
    if (s->pending.empty()) return;
    cudaStreamSynchronize(s->st);
    for (auto& p : s->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            s->ms[p.kid] += ms;
            s->launches[p.kid] += 1;
        }
        s->ev_free.push_back(p.a);
        s->ev_free.push_back(p.b);
    }
    s->pending.clear();
}

void hook_begin(void* ctx, int kid) {
    evp_state* s = static_cast<evp_state*>(ctx);
    if (s->nvtx) nvtxRangePushA(KERNEL_NAMES[kid]);
    if (!s->timing) return;
    s->cur_start = get_event(s);
    cudaEventRecord(s->cur_start, s->st);
}

void hook_end(void* ctx, int kid) {
    evp_state* s = static_cast<evp_state*>(ctx);
    if (s->timing) {
        cudaEvent_t e = get_event(s);
        cudaEventRecord(e, s->st);
        s->pending.push_back({kid, s->cur_start, e});
        if (s->pending.size() >= 2048) flush_timing(s);
    }
    if (s->nvtx) nvtxRangePop();
}

// An NVTX range for the lifetime of the object when the state's ranges are on
struct NvtxScope {
    bool on;
    NvtxScope(const evp_state* s, const char* name) : on(s && s->nvtx) {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxScope() {
        if (on) nvtxRangePop();
    }
};

TimingHook hook_of(evp_state* s) {
    TimingHook h;
    h.begin = (s->timing || s->nvtx) ? hook_begin : nullptr;
    h.end = (s->timing || s->nvtx) ? hook_end : nullptr;
    h.pdl = s->pdl;
    h.ctx = s;
    return h;
}

int validate(const evp_grid* g, evp_model model, const evp_params* p) {
    if (!g || !p) return fail(EVP_ERR_ARG, "null grid or params");
    auto fft_ok = [](int n) { return n >= 8 && n <= 512 && is_2a3b(n); };
    if (!fft_ok(g->nx) || (g->nx % 2) != 0) return fail(EVP_ERR_ARG, "nx must be even, 2^a 3^b, 8..512");
    if (!fft_ok(g->nz)) return fail(EVP_ERR_ARG, "nz must be 2^a 3^b, 8..512");
    if (g->walls_y) {
        if (g->ny < 4 || g->ny > 512) return fail(EVP_ERR_ARG, "ny with walls must be 4..512");
    } else if (!fft_ok(g->ny)) {
        return fail(EVP_ERR_ARG, "periodic ny must be 2^a 3^b, 8..512");
    }
    if (!(g->lx > 0) || !(g->ly > 0) || !(g->lz > 0)) return fail(EVP_ERR_ARG, "box lengths must be positive");
    if (model < EVP_NEWTONIAN || model > EVP_NEO_HOOKEAN) return fail(EVP_ERR_ARG, "unknown model");
    if (!(p->Re > 0)) return fail(EVP_ERR_ARG, "Re must be positive");
    if (!(p->beta >= 0 && p->beta <= 1)) return fail(EVP_ERR_ARG, "beta must be in [0, 1]");
    if (model != EVP_NEWTONIAN && !(p->Wi > 0)) return fail(EVP_ERR_ARG, "Wi must be positive");
    if (model == EVP_FENE_P && !(p->L2 > 3)) return fail(EVP_ERR_ARG, "FENE-P needs L2 > 3");
    if (model == EVP_SARAMITO && !(p->Bi >= 0)) return fail(EVP_ERR_ARG, "Bi must be >= 0");
    if (!(p->art_diff >= 0) || !(p->art_diff < 1e300)) return fail(EVP_ERR_ARG, "art_diff must be finite and >= 0");
    if (p->precision != EVP_FP64 && p->precision != EVP_FP32) return fail(EVP_ERR_ARG, "bad precision");
    if (p->integrator != EVP_RK3 && p->integrator != EVP_AB2) return fail(EVP_ERR_ARG, "unknown integrator");
    if (p->integrator == EVP_AB2) {
        if (p->penalization) return fail(EVP_ERR_ARG, "volume penalisation is part of the RK3 step only");
        if (p->dpdx != 0.0 || p->abc_amp != 0.0)
            return fail(EVP_ERR_ARG, "the AB2 two-phase step takes no dpdx or ABC forcing");
        if (!(p->rho_ratio >= 0)) return fail(EVP_ERR_ARG, "rho_ratio must be >= 0 (0: Boussinesq)");
        if (!(p->mu_ratio > 0) || !(p->ls_eps_cells > 0) || !(p->sigma >= 0) || p->reinit_every < 0 ||
            p->reinit_iters < 0)
            return fail(EVP_ERR_ARG, "bad two-phase parameters (mu_ratio, ls_eps_cells, sigma, reinit)");
        if (p->ls_mass_iters < 0 || p->ls_mass_iters > 50) return fail(EVP_ERR_ARG, "ls_mass_iters must be 0..50");
    } else if (p->ls_mass_iters != 0) {
        return fail(EVP_ERR_ARG, "the level-set mass correction is part of the AB2 two-phase step");
    }
    if (p->thomas_fp64 != 0 && p->thomas_fp64 != 1) return fail(EVP_ERR_ARG, "thomas_fp64 must be 0 or 1");
    if (p->soft_particles) {
        if (p->soft_particles != 1) return fail(EVP_ERR_ARG, "soft_particles must be 0 or 1");
        if (model != EVP_NEO_HOOKEAN) return fail(EVP_ERR_ARG, "soft particles need the neo-Hookean model");
        if (p->integrator != EVP_RK3) return fail(EVP_ERR_ARG, "soft particles are part of the RK3 step");
    }
    if (p->viscous_implicit) {
        if (p->viscous_implicit != 1) return fail(EVP_ERR_ARG, "viscous_implicit must be 0 or 1");
        if (p->integrator != EVP_RK3) return fail(EVP_ERR_ARG, "the implicit viscous option is part of the RK3 step");
        if (p->penalization) return fail(EVP_ERR_ARG, "the implicit viscous option does not combine with penalization");
    }
    return EVP_OK;
}

struct Layout {
    size_t off[64];
    int n = 0;
    size_t total = 0;
    size_t add(size_t bytes) {
        size_t o = total;
        off[n++] = o;
        total += align_up(bytes);
        return o;
    }
};

// Build the arena layout; returns total bytes.  With base != null also assigns pointers.
size_t plan(evp_state* s, char* base) {
    const evp_grid& g = s->g;
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    const size_t e = s->elt;
    const int nxh = g.nx / 2 + 1;
    Layout L;
    auto P = [&](size_t bytes) -> void* { size_t o = L.add(bytes); return base ? base + o : nullptr; };
    for (int b = 0; b < 2; ++b) {
        void* u = P(N * e);
        void* v = P(N * e);
        void* w = P(N * e);
        if (base) { s->U[b] = u; s->V[b] = v; s->W[b] = w; }
    }
    for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 6; ++c) {
            void* p = P(N * e);
            if (base) s->B[b][c] = p;
        }
    for (int c = 0; c < 6; ++c) { void* p = P(N * e); if (base) s->RT[c] = p; }
    for (int c = 0; c < 3; ++c) { void* p = P(N * e); if (base) s->NH[c] = p; }
    const bool sum_stress = s->model != EVP_NEWTONIAN && s->prm.integrator != EVP_AB2 && !s->prm.soft_particles;
    for (int c = 0; c < 6; ++c) {
        void* p = sum_stress ? P(N * e) : nullptr;
        if (base) s->S[c] = p;
    }
    void* p = P(N * e);
    void* psi = P(N * e);
    void* spec = P((size_t)nxh * g.ny * g.nz * 2 * e);
    void* twx = P((size_t)g.nx * 2 * e);
    void* twy = P((size_t)g.ny * 2 * e);
    void* twz = P((size_t)g.nz * 2 * e);
    void* lamx = P((size_t)nxh * e);
    void* lamy = P((size_t)g.ny * e);
    void* lamz = P((size_t)g.nz * e);
    void* trig = P((size_t)2 * (g.nx + g.ny + g.nz) * e);
    void* thm = g.walls_y ? P((size_t)(g.nz / 2 + 1) * g.ny * nxh * sizeof(double2)) : nullptr;
    void* thd = g.walls_y ? P((size_t)2 * nxh * g.ny * g.nz * sizeof(double)) : nullptr;
    const bool ab2 = s->prm.integrator == EVP_AB2;
    void* ls[12] = {nullptr};
    if (ab2)
        for (int q = 0; q < 12; ++q) ls[q] = P(N * e);   // phi, phi0, phiA, phiB, H, n(3), f(3), p^{n-1}
    const size_t nparts = (size_t)((g.nx + 31) / 32) * ((g.ny + 7) / 8) * g.nz;
    void* parts = ab2 ? P(nparts * sizeof(double)) : nullptr;
    void* sol[3] = {nullptr, nullptr, nullptr};
    if (s->prm.penalization)
        for (int q = 0; q < 3; ++q) sol[q] = P(N * e);
    void* mean = ab2 ? P(sizeof(double)) : nullptr;
    void* mass = (ab2 && s->prm.ls_mass_iters > 0) ? P((2 * nparts + 2) * sizeof(double)) : nullptr;
    void* phs[3] = {nullptr, nullptr, nullptr};
    if (s->prm.soft_particles)
        for (int q = 0; q < 3; ++q) phs[q] = P(N * e);
    void* helm[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    if (s->prm.viscous_implicit && g.walls_y)
        for (int k = 0; k < 3; ++k)
            for (int q = 0; q < 2; ++q) helm[k][q] = P((size_t)(g.nz / 2 + 1) * g.ny * nxh * sizeof(double2));
    void* st = P(sizeof(unsigned));
    void* md = P(sizeof(unsigned long long));
    void* dg = P((evp::DIAG_BLOCKS + 1) * sizeof(evp::DiagPart));
    if (base) {
        s->P = p; s->PSI = psi; s->spec = spec;
        s->twx = twx; s->twy = twy; s->twz = twz;
        s->lamx = lamx; s->lamy = lamy; s->lamz = lamz; s->trig = trig;
        s->thomas_m = static_cast<double2*>(thm);
        s->thomas_d = static_cast<double*>(thd);
        s->d_status = static_cast<unsigned*>(st);
        s->d_maxdiv = static_cast<unsigned long long*>(md);
        s->diag = dg;
        s->ab2 = ab2;
        s->PHI = ls[0];
        s->PHI0 = ls[1];
        s->PHIA = ls[2];
        s->PHIB = ls[3];
        s->HF = ls[4];
        for (int q = 0; q < 3; ++q) {
            s->NRM[q] = ls[5 + q];
            s->FC[q] = ls[8 + q];
        }
        s->POLD = ls[11];
        s->partials = static_cast<double*>(parts);
        for (int q = 0; q < 3; ++q) s->SOL[q] = sol[q];
        s->mean_1mH = static_cast<double*>(mean);
        s->mass = static_cast<double*>(mass);
        s->PHS[0] = phs[0];
        s->PHS[1] = phs[1];
        s->PHSH = phs[2];
        for (int k = 0; k < 3; ++k)
            for (int q = 0; q < 2; ++q) s->helm[k][q] = static_cast<double2*>(helm[k][q]);
        s->helm_dt = -1.0;
    }
    return L.total;
}

template <typename T>
__global__ void k_fill(T* p, size_t n, T v) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

template <typename T>
std::vector<T> to_t(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

template <typename T>
int upload_tables(evp_state* s) {
    const evp_grid& g = s->g;
    const double dx = g.lx / g.nx, dy = g.ly / g.ny, dz = g.lz / g.nz;
    const int nxh = g.nx / 2 + 1;
    const double twopi = 6.283185307179586476925286766559;
    auto tw = [&](int n) {
        std::vector<double> v(2 * n);
        for (int m = 0; m < n; ++m) {
            v[2 * m] = std::cos(twopi * m / n);
            v[2 * m + 1] = -std::sin(twopi * m / n);
        }
        return v;
    };
    auto lam = [&](int n, int cnt, double h) {
        std::vector<double> v(cnt);
        for (int m = 0; m < cnt; ++m) v[m] = (2.0 - 2.0 * std::cos(twopi * m / n)) / (h * h);
        return v;
    };
    auto put = [&](void* dst, const std::vector<double>& v) -> cudaError_t {
        std::vector<T> t = to_t<T>(v);
        return cudaMemcpyAsync(dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, s->st);
    };
    CK(put(s->twx, tw(g.nx)));
    CK(put(s->twy, tw(g.ny)));
    CK(put(s->twz, tw(g.nz)));
    std::vector<double> lx = lam(g.nx, nxh, dx), ly = lam(g.ny, g.ny, dy), lz = lam(g.nz, g.nz, dz);
    CK(put(s->lamx, lx));
    CK(put(s->lamy, ly));
    CK(put(s->lamz, lz));
    // ABC forcing tables sin/cos(k x_i), (k y_j), (k z_k) at cell centres
    {
        const double k = s->prm.abc_k;
        const double y0 = g.walls_y ? -0.5 * g.ly : 0.0;
        std::vector<double> t;
        for (int i = 0; i < g.nx; ++i) t.push_back(std::sin(k * (i + 0.5) * dx));
        for (int i = 0; i < g.nx; ++i) t.push_back(std::cos(k * (i + 0.5) * dx));
        for (int j = 0; j < g.ny; ++j) t.push_back(std::sin(k * (y0 + (j + 0.5) * dy)));
        for (int j = 0; j < g.ny; ++j) t.push_back(std::cos(k * (y0 + (j + 0.5) * dy)));
        for (int q = 0; q < g.nz; ++q) t.push_back(std::sin(k * (q + 0.5) * dz));
        for (int q = 0; q < g.nz; ++q) t.push_back(std::cos(k * (q + 0.5) * dz));
        CK(put(s->trig, t));
    }
    if (g.walls_y) {
        // Thomas table (m_j, c'_j) per (kz <= nz/2, kx), built in FP64
        const std::vector<double> M = thomas_table(g.ny, g.nz, nxh, dy, lx, lam(g.nz, g.nz / 2 + 1, dz));
        if (sizeof(T) == 4 && !s->prm.thomas_fp64) {
            // single-precision states sweep in double-single arithmetic (k_thomas)
            const std::vector<float> F = thomas_table_ds(M);
            CK(cudaMemcpyAsync(s->thomas_m, F.data(), F.size() * sizeof(float), cudaMemcpyHostToDevice, s->st));
        } else {
            CK(cudaMemcpyAsync(s->thomas_m, M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice, s->st));
        }
    }
    return cudaStreamSynchronize(s->st) == cudaSuccess ? EVP_OK : cuda_fail(cudaGetLastError(), "tables");
}




template <typename T>
int run_poisson(evp_state* s, const T* Us, const T* Vs, const T* Ws, const T* rhs, double rscale, T* psi) {
    PoissonArgs<T> a;
    a.Us = Us;
    a.Vs = Vs;
    a.Ws = Ws;
    a.rhs = rhs;
    a.rscale = T(rscale);
    a.spec = static_cast<typename Cplx<T>::type*>(s->spec);
    a.psi = psi;
    a.norm = poisson_norm<T>(s);
    a.out_scale = s->g.walls_y ? T(a.norm) : T(1);
    a.scratch = s->thomas_d;
    cudaError_t e = launch_poisson<T>(geo_of<T>(s), tables_of<T>(s), a, s->st, hook_of(s));
    return e == cudaSuccess ? EVP_OK : cuda_fail(e, "poisson");
}

// Implicit viscous option: field <- solution of x - c lap(x) = field for one
// velocity component (kind_v: the v rule), in place through the spectral buffer
template <typename T>
int run_helmholtz(evp_state* s, T* field, double c, int k, bool kind_v) {
    PoissonArgs<T> a;
    a.Us = a.Vs = a.Ws = nullptr;
    a.rhs = field;
    a.rscale = T(1);
    a.spec = static_cast<typename Cplx<T>::type*>(s->spec);
    a.psi = field;
    a.norm = poisson_norm<T>(s);
    a.out_scale = s->g.walls_y ? T(a.norm) : T(1);
    a.scratch = s->thomas_d;
    if (s->g.walls_y) {
        const double dy = s->g.ly / s->g.ny;
        a.ttab = s->helm[k][kind_v ? 1 : 0];
        a.tsub = -c / (dy * dy);
    } else {
        a.hcoef = T(c);
    }
    cudaError_t e = launch_poisson<T>(geo_of<T>(s), tables_of<T>(s), a, s->st, hook_of(s));
    return e == cudaSuccess ? EVP_OK : cuda_fail(e, "helmholtz");
}

// Host: (re)build the Helmholtz Thomas tables of the three substeps for this dt
int prepare_helmholtz(evp_state* s, double dt) {
    if (!s->prm.viscous_implicit || !s->g.walls_y || s->helm_dt == dt) return EVP_OK;
    const evp_grid& g = s->g;
    const int nxh = g.nx / 2 + 1;
    const double dx = g.lx / g.nx, dy = g.ly / g.ny, dz = g.lz / g.nz;
    auto lam = [&](int n, int cnt, double h) {
        std::vector<double> v(cnt);
        for (int m = 0; m < cnt; ++m) v[m] = (2.0 - 2.0 * std::cos(2.0 * M_PI * m / n)) / (h * h);
        return v;
    };
    const std::vector<double> lx = lam(g.nx, nxh, dx), lz = lam(g.nz, g.nz / 2 + 1, dz);
    const double mu_s = s->prm.beta / s->prm.Re;
    static const double RK3_ALPHA_H[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
    CK(cudaStreamSynchronize(s->st));
    for (int k = 0; k < 3; ++k)
        for (int q = 0; q < 2; ++q) {
            const std::vector<double> M = helmholtz_table(g.ny, g.nz, nxh, dy, lx, lz, RK3_ALPHA_H[k] * dt * mu_s, q == 1);
            if (s->fp32 && !s->prm.thomas_fp64) {
                const std::vector<float> F = thomas_table_ds(M);
                CK(cudaMemcpy(s->helm[k][q], F.data(), F.size() * sizeof(float), cudaMemcpyHostToDevice));
            } else {
                CK(cudaMemcpy(s->helm[k][q], M.data(), M.size() * sizeof(double), cudaMemcpyHostToDevice));
            }
        }
    s->helm_dt = dt;
    return EVP_OK;
}

template <typename T>
int run_correct(evp_state* s, const T* Us, const T* Vs, const T* Ws, T* U, T* V, T* W, T* P, double coef,
                bool p_replace = false) {
    CorrectArgs<T> a;
    a.Us = Us;
    a.Vs = Vs;
    a.Ws = Ws;
    a.psi = static_cast<const T*>(s->PSI);
    a.U = U;
    a.V = V;
    a.W = W;
    a.P = P;
    a.p_replace = p_replace ? 1 : 0;
    a.coef = T(coef);
    a.status = s->d_status;
    cudaError_t e = launch_correct<T>(geo_of<T>(s), a, s->st, hook_of(s));
    return e == cudaSuccess ? EVP_OK : cuda_fail(e, "correct");
}

// One RK3 substep; last_in_step: the third substep of evp_step (no history written).
template <typename T>
int substep_t(evp_state* s, double dt, int k, bool last_in_step) {
    const double al = RK_ALPHA[k], ze = RK_ZETA[k], xi = RK_XI[k];
    const bool stress = s->model != EVP_NEWTONIAN;
    const int cu = s->cu, cb = s->cb;
    const Geo<T> g = geo_of<T>(s);
    const TimingHook th = hook_of(s);
    const bool read_hist = xi != 0.0, write_hist = !last_in_step;
    if (stress) {
        StressArgs<T> a;
        a.U = static_cast<const T*>(s->U[cu]);
        a.V = static_cast<const T*>(s->V[cu]);
        a.W = static_cast<const T*>(s->W[cu]);
        for (int c = 0; c < 6; ++c) {
            a.B[c] = static_cast<const T*>(s->B[cb][c]);
            a.Bn[c] = static_cast<T*>(s->B[1 - cb][c]);
            a.RT[c] = static_cast<T*>(s->RT[c]);
        }
        a.dt_zeta = T(dt * ze);
        a.dt_xi = T(dt * xi);
        a.read_hist = read_hist;
        a.write_hist = write_hist;
        a.rhs_only = 0;
        a.status = s->d_status;
        a.H = nullptr;
        a.mu_p1 = a.mu_p2 = T(0);
        for (int c = 0; c < 6; ++c) a.S[c] = static_cast<T*>(s->S[c]);
        cudaError_t e = launch_stress<T>(g, s->mc, a, s->st, th);
        if (e != cudaSuccess) return cuda_fail(e, "stress kernel");
    }
    {
        MomentumArgs<T> a;
        a.status = s->d_status;
        a.U = static_cast<const T*>(s->U[cu]);
        a.V = static_cast<const T*>(s->V[cu]);
        a.W = static_cast<const T*>(s->W[cu]);
        a.P = static_cast<const T*>(s->P);
        for (int c = 0; c < 6; ++c) {
            a.Bo[c] = static_cast<const T*>(s->B[cb][c]);
            a.Bn[c] = static_cast<const T*>(s->B[stress ? 1 - cb : cb][c]);
        }
        a.Us = static_cast<T*>(s->U[1 - cu]);
        a.Vs = static_cast<T*>(s->V[1 - cu]);
        a.Ws = static_cast<T*>(s->W[1 - cu]);
        for (int c = 0; c < 3; ++c) a.NH[c] = static_cast<T*>(s->NH[c]);
        a.dt = T(dt);
        a.zeta = T(ze);
        a.xi = T(xi);
        a.alpha = T(al);
        a.read_hist = read_hist;
        a.write_hist = write_hist;
        a.has_stress = stress;
        a.dpdx = T(s->prm.dpdx);
        a.abc_amp = T(s->prm.abc_amp);
        a.trig = s->prm.abc_amp != 0.0 ? static_cast<const T*>(s->trig) : nullptr;
        for (int q = 0; q < 3; ++q) a.solid[q] = static_cast<const T*>(s->SOL[q]);
        a.cn = s->prm.viscous_implicit ? 1 : 0;
        if (stress)
            for (int c = 0; c < 6; ++c) a.S[c] = static_cast<const T*>(s->S[c]);
        if (s->prm.soft_particles) {
            // solid fraction phi^k from phi^{k-1} with u^{k-1}, then tau = phi_s G (B - I)
            PhisArgs<T> f;
            f.U = static_cast<const T*>(s->U[cu]);
            f.V = static_cast<const T*>(s->V[cu]);
            f.W = static_cast<const T*>(s->W[cu]);
            f.phi = static_cast<const T*>(s->PHS[cb]);
            f.phin = static_cast<T*>(s->PHS[1 - cb]);
            f.hist = static_cast<T*>(s->PHSH);
            f.dt_zeta = T(dt * ze);
            f.dt_xi = T(dt * xi);
            f.read_hist = read_hist;
            f.write_hist = write_hist;
            if (cudaError_t e = launch_phis<T>(g, f, s->st, th)) return cuda_fail(e, "solid fraction");
            a.phis_o = f.phi;
            a.phis_n = f.phin;
        }
        cudaError_t e = launch_momentum<T>(g, s->mc, a, s->st, th);
        if (e != cudaSuccess) return cuda_fail(e, "momentum kernel");
    }
    if (s->prm.viscous_implicit) {
        // Helmholtz solve per component: u* - alpha dt mu_s lap u* = rhs (Reading 18)
        const double c = al * dt * s->mc.mu_s;
        T* star[3] = {static_cast<T*>(s->U[1 - cu]), static_cast<T*>(s->V[1 - cu]), static_cast<T*>(s->W[1 - cu])};
        for (int q = 0; q < 3; ++q)
            if (int r = run_helmholtz<T>(s, star[q], c, k, q == 1)) return r;
    }
    if (s->n_part > 0) {
        // discrete-forcing IBM of the rigid particles: u* -> u** (Eqs. IBM, CoVe2)
        IbmArgs<T> b;
        b.U[0] = static_cast<T*>(s->U[1 - cu]);
        b.U[1] = static_cast<T*>(s->V[1 - cu]);
        b.U[2] = static_cast<T*>(s->W[1 - cu]);
        b.off = s->i_off;
        b.owner = s->i_owner;
        b.start = s->i_start;
        b.dvl = s->i_dvl;
        b.centre = s->i_centre;
        b.pvel = s->i_vel;
        b.pomg = s->i_omg;
        b.Facc = s->i_Facc;
        b.dF = s->i_dF;
        b.pforce = s->i_force;
        b.pvel_w = s->i_vel;
        b.pomg_w = s->i_omg;
        b.prad = s->i_rad;
        b.pdens = s->i_dens;
        b.I0 = s->i_int;
        b.I1 = s->i_int + 6 * s->n_part;
        b.nl = s->n_lag;
        b.np = s->n_part;
        b.nx = s->g.nx;
        b.ny = s->g.ny;
        b.nz = s->g.nz;
        b.walls = s->g.walls_y;
        b.any_free = s->any_free;
        b.dx = s->g.lx / s->g.nx;
        b.dy = s->g.ly / s->g.ny;
        b.dz = s->g.lz / s->g.nz;
        b.y0 = s->g.walls_y ? -0.5 * s->g.ly : 0.0;
        b.lx = s->g.lx;
        b.ly = s->g.ly;
        b.lz = s->g.lz;
        b.dts = 2.0 * al * dt;
        b.gravity = s->prm.gravity;
        const T* uold[3] = {static_cast<const T*>(s->U[cu]), static_cast<const T*>(s->V[cu]),
                            static_cast<const T*>(s->W[cu])};
        cudaError_t e = launch_ibm<T>(b, uold, s->ibm_iters, s->st, th);
        if (e != cudaSuccess) return cuda_fail(e, "ibm");
    }
    const double coef = 2.0 * al * dt;
    int r = run_poisson<T>(s, static_cast<const T*>(s->U[1 - cu]), static_cast<const T*>(s->V[1 - cu]),
                           static_cast<const T*>(s->W[1 - cu]), nullptr, 1.0 / coef, static_cast<T*>(s->PSI));
    if (r) return r;
    r = run_correct<T>(s, static_cast<const T*>(s->U[1 - cu]), static_cast<const T*>(s->V[1 - cu]),
                       static_cast<const T*>(s->W[1 - cu]), static_cast<T*>(s->U[cu]), static_cast<T*>(s->V[cu]),
                       static_cast<T*>(s->W[cu]), static_cast<T*>(s->P), coef);
    if (r) return r;
    if (stress) s->cb = 1 - cb;
    return EVP_OK;
}

// One two-phase AB2 step (Secs. 3.2.1-3.2.2): level set, re-distancing when due,
// interface force, B (Eq. ab2tau) and u* (Eq. ab2), projection with dt.
template <typename T>
int ab2_step_t(evp_state* s, double dt) {
    const Geo<T> g = geo_of<T>(s);
    const TimingHook th = hook_of(s);
    const evp_params& p = s->prm;
    const int cu = s->cu, cb = s->cb;
    const double dx = s->g.lx / s->g.nx;
    const bool stress = s->model != EVP_NEWTONIAN;
    auto stage = [&](const void* phin, const void* phis, void* out, double a, double b, bool reinit, double h) {
        LsArgs<T> L;
        L.U = static_cast<const T*>(s->U[cu]);
        L.V = static_cast<const T*>(s->V[cu]);
        L.W = static_cast<const T*>(s->W[cu]);
        L.phin = static_cast<const T*>(phin);
        L.phis = static_cast<const T*>(phis);
        L.phi0 = static_cast<const T*>(s->PHI0);
        L.out = static_cast<T*>(out);
        L.pt_a = T(a);
        L.pt_b = T(b);
        L.dt = T(h);
        L.h = T(dx);
        return launch_ls_stage<T>(g, L, reinit, s->st, th);
    };
    // mass correction (Reading 17): shift of phi restoring the drop volume of the first step
    const size_t np_mass = iface_partials(g);
    MassArgs<T> M;
    M.phi = static_cast<T*>(s->PHI);
    M.eps = T(p.ls_eps_cells * dx);
    M.partials = s->mass;
    M.v0 = s->mass ? s->mass + 2 * np_mass : nullptr;
    M.d = s->mass ? s->mass + 2 * np_mass + 1 : nullptr;
    M.dv = (s->g.lx / s->g.nx) * (s->g.ly / s->g.ny) * (s->g.lz / s->g.nz);
    cudaError_t e;
    if (p.ls_mass_iters > 0 && s->nstep == 0)
        if ((e = launch_mass_correct<T>(g, M, 0, 0, s->st, th)) != cudaSuccess) return cuda_fail(e, "mass correction");
    // 1. level set: TVD-RK3 with u^n; the third stage writes phi in place
    if ((e = stage(s->PHI, s->PHI, s->PHIA, 0.0, 1.0, false, dt)) != cudaSuccess) return cuda_fail(e, "level set");
    if ((e = stage(s->PHI, s->PHIA, s->PHIB, 0.75, 0.25, false, dt)) != cudaSuccess) return cuda_fail(e, "level set");
    if ((e = stage(s->PHI, s->PHIB, s->PHI, 1.0 / 3.0, 2.0 / 3.0, false, dt)) != cudaSuccess)
        return cuda_fail(e, "level set");
    if (p.reinit_every > 0 && (s->nstep + 1) % p.reinit_every == 0 && p.reinit_iters > 0) {
        CK(cudaMemcpyAsync(s->PHI0, s->PHI, s->N * sizeof(T), cudaMemcpyDeviceToDevice, s->st));
        const double dtau = 0.5 * dx;
        for (int it = 0; it < p.reinit_iters; ++it) {
            if ((e = stage(s->PHI, s->PHI, s->PHIA, 0.0, 1.0, true, dtau)) != cudaSuccess) return cuda_fail(e, "reinit");
            if ((e = stage(s->PHI, s->PHIA, s->PHIB, 0.75, 0.25, true, dtau)) != cudaSuccess)
                return cuda_fail(e, "reinit");
            if ((e = stage(s->PHI, s->PHIB, s->PHI, 1.0 / 3.0, 2.0 / 3.0, true, dtau)) != cudaSuccess)
                return cuda_fail(e, "reinit");
        }
    }
    if (p.ls_mass_iters > 0)
        if ((e = launch_mass_correct<T>(g, M, 1, p.ls_mass_iters, s->st, th)) != cudaSuccess)
            return cuda_fail(e, "mass correction");
    // 2. H, normals, interface force at n+1
    {
        IfaceArgs<T> I;
        I.phi = static_cast<const T*>(s->PHI);
        I.H = static_cast<T*>(s->HF);
        for (int q = 0; q < 3; ++q) {
            I.n[q] = static_cast<T*>(s->NRM[q]);
            I.f[q] = static_cast<T*>(s->FC[q]);
        }
        I.partials = s->partials;
        I.mean_1mH = s->mean_1mH;
        I.eps = T(p.ls_eps_cells * dx);
        I.sigma = T(p.sigma);
        I.drho_g = T(p.rho_ratio > 0 ? 0.0 : p.drho_g);
        if ((e = launch_interface<T>(g, I, s->st, th)) != cudaSuccess) return cuda_fail(e, "interface");
    }
    const bool first = s->nstep == 0;
    const double w1 = first ? 1.0 : 1.5, w0 = first ? 0.0 : -0.5;
    const double mu0 = 1.0 / p.Re;
    const T mp1 = T((1.0 - p.beta) * mu0), mp2 = T(0);
    // 3. B^{n+1} = B^n + dt (w1 RT^n + w0 RT^{n-1})
    if (stress) {
        StressArgs<T> a;
        a.U = static_cast<const T*>(s->U[cu]);
        a.V = static_cast<const T*>(s->V[cu]);
        a.W = static_cast<const T*>(s->W[cu]);
        for (int c = 0; c < 6; ++c) {
            a.B[c] = static_cast<const T*>(s->B[cb][c]);
            a.Bn[c] = static_cast<T*>(s->B[1 - cb][c]);
            a.RT[c] = static_cast<T*>(s->RT[c]);
        }
        a.dt_zeta = T(dt * w1);
        a.dt_xi = T(dt * w0);
        a.read_hist = !first;
        a.write_hist = 1;
        a.rhs_only = 0;
        a.status = s->d_status;
        a.H = static_cast<const T*>(s->HF);
        a.mu_p1 = mp1;
        a.mu_p2 = mp2;
        if ((e = launch_stress<T>(g, s->mc, a, s->st, th)) != cudaSuccess) return cuda_fail(e, "stress kernel");
    }
    // 4. u* = u^n + dt (w1 RU^n + w0 RU^{n-1}), tau^n from B^n with mu_p(H^{n+1})
    {
        MomAB2Args<T> m;
        m.U = static_cast<const T*>(s->U[cu]);
        m.V = static_cast<const T*>(s->V[cu]);
        m.W = static_cast<const T*>(s->W[cu]);
        for (int c = 0; c < 6; ++c) m.B[c] = static_cast<const T*>(s->B[cb][c]);
        m.H = static_cast<const T*>(s->HF);
        for (int q = 0; q < 3; ++q) {
            m.f[q] = static_cast<const T*>(s->FC[q]);
            m.NH[q] = static_cast<T*>(s->NH[q]);
        }
        m.Us = static_cast<T*>(s->U[1 - cu]);
        m.Vs = static_cast<T*>(s->V[1 - cu]);
        m.Ws = static_cast<T*>(s->W[1 - cu]);
        m.w1dt = T(dt * w1);
        m.w0dt = T(dt * w0);
        m.read_hist = !first;
        m.mu_s1 = T(p.beta * mu0);
        m.mu_s2 = T(p.mu_ratio * mu0);
        m.mu_p1 = mp1;
        m.mu_p2 = mp2;
        m.inv_lam = T(s->mc.inv_lam);
        m.L2 = T(s->mc.L2);
        m.a_fene = T(s->mc.a_fene);
        m.rho_ratio = T(p.rho_ratio);
        m.gravity = T(p.gravity);
        m.mean_1mH = s->mean_1mH;
        if ((e = launch_momentum_ab2<T>(g, s->model, m, s->st, th)) != cudaSuccess)
            return cuda_fail(e, "momentum kernel");
    }
    if (p.rho_ratio > 0) {
        // 5'. constant-coefficient split projection (Eqs. poisson-LS, projection-LS)
        if (first) CK(cudaMemcpyAsync(s->POLD, s->P, s->N * sizeof(T), cudaMemcpyDeviceToDevice, s->st));
        SplitArgs<T> q;
        q.Us = static_cast<const T*>(s->U[1 - cu]);
        q.Vs = static_cast<const T*>(s->V[1 - cu]);
        q.Ws = static_cast<const T*>(s->W[1 - cu]);
        q.P = static_cast<const T*>(s->P);
        q.Pold = static_cast<const T*>(s->POLD);
        q.H = static_cast<const T*>(s->HF);
        q.R = static_cast<T*>(s->PSI);
        q.U = static_cast<T*>(s->U[cu]);
        q.V = static_cast<T*>(s->V[cu]);
        q.W = static_cast<T*>(s->W[cu]);
        q.rho_ratio = T(p.rho_ratio);
        q.rho0 = T(p.rho_ratio < 1.0 ? p.rho_ratio : 1.0);
        q.dt = T(dt);
        q.status = s->d_status;
        if ((e = launch_split_rhs<T>(g, q, s->st, th)) != cudaSuccess) return cuda_fail(e, "split rhs");
        int r = run_poisson<T>(s, nullptr, nullptr, nullptr, static_cast<const T*>(s->PSI), 1.0, static_cast<T*>(s->PSI));
        if (r) return r;
        if ((e = launch_split_correct<T>(g, q, s->st, th)) != cudaSuccess) return cuda_fail(e, "split correct");
        // rotate: p^{n-1} <- p^n, p^n <- p^{n+1}; the old p^{n-1} buffer becomes scratch
        void* old = s->POLD;
        s->POLD = s->P;
        s->P = s->PSI;
        s->PSI = old;
        if (stress) s->cb = 1 - cb;
        s->nstep += 1;
        return EVP_OK;
    }
    // 5. projection with dt: p^{n+1} = psi
    int r = run_poisson<T>(s, static_cast<const T*>(s->U[1 - cu]), static_cast<const T*>(s->V[1 - cu]),
                           static_cast<const T*>(s->W[1 - cu]), nullptr, 1.0 / dt, static_cast<T*>(s->PSI));
    if (r) return r;
    r = run_correct<T>(s, static_cast<const T*>(s->U[1 - cu]), static_cast<const T*>(s->V[1 - cu]),
                       static_cast<const T*>(s->W[1 - cu]), static_cast<T*>(s->U[cu]), static_cast<T*>(s->V[cu]),
                       static_cast<T*>(s->W[cu]), static_cast<T*>(s->P), dt, true);
    if (r) return r;
    if (stress) s->cb = 1 - cb;
    s->nstep += 1;
    return EVP_OK;
}

void* field_ptr(evp_state* s, int f) {
    if (f == EVP_U) return s->U[s->cu];
    if (f == EVP_V) return s->V[s->cu];
    if (f == EVP_W) return s->W[s->cu];
    if (f == EVP_P) return s->P;
    if (f >= EVP_BXX && f <= EVP_BZZ) return s->B[s->cb][f - EVP_BXX];
    if (f >= EVP_RT_XX && f < EVP_RT_XX + 6) return s->RT[f - EVP_RT_XX];
    if (f >= EVP_NH_X && f < EVP_NH_X + 3) return s->NH[f - EVP_NH_X];
    if (f == EVP_PSI) return s->PSI;
    if (f == EVP_PHI) return s->ab2 ? s->PHI : (s->prm.soft_particles ? s->PHS[s->cb] : nullptr);
    if (f >= EVP_SOLID_X && f <= EVP_SOLID_Z) return s->SOL[f - EVP_SOLID_X];
    return nullptr;
}

template <typename T>
int init_fields(evp_state* s) {
    const size_t N = s->N;
    for (int b = 0; b < 2; ++b) {
        CK(cudaMemsetAsync(s->U[b], 0, N * sizeof(T), s->st));
        CK(cudaMemsetAsync(s->V[b], 0, N * sizeof(T), s->st));
        CK(cudaMemsetAsync(s->W[b], 0, N * sizeof(T), s->st));
        for (int c = 0; c < 6; ++c) {
            const bool diag = (c == 0 || c == 3 || c == 5);
            if (diag) {
                k_fill<T><<<(unsigned)((N + 255) / 256), 256, 0, s->st>>>(static_cast<T*>(s->B[b][c]), N, T(1));
                CK(cudaGetLastError());
            } else {
                CK(cudaMemsetAsync(s->B[b][c], 0, N * sizeof(T), s->st));
            }
        }
    }
    for (int c = 0; c < 6; ++c) CK(cudaMemsetAsync(s->RT[c], 0, N * sizeof(T), s->st));
    for (int c = 0; c < 3; ++c) CK(cudaMemsetAsync(s->NH[c], 0, N * sizeof(T), s->st));
    CK(cudaMemsetAsync(s->P, 0, N * sizeof(T), s->st));
    CK(cudaMemsetAsync(s->PSI, 0, N * sizeof(T), s->st));
    for (int q = 0; q < 3; ++q)
        if (s->SOL[q]) CK(cudaMemsetAsync(s->SOL[q], 0, N * sizeof(T), s->st));
    if (s->prm.soft_particles) {
        CK(cudaMemsetAsync(s->PHS[0], 0, N * sizeof(T), s->st));
        CK(cudaMemsetAsync(s->PHS[1], 0, N * sizeof(T), s->st));
        CK(cudaMemsetAsync(s->PHSH, 0, N * sizeof(T), s->st));
    }
    if (s->ab2) {
        void* z[] = {s->PHI, s->PHI0, s->PHIA, s->PHIB, s->HF, s->NRM[0], s->NRM[1], s->NRM[2],
                     s->FC[0], s->FC[1], s->FC[2], s->POLD};
        for (void* q : z) CK(cudaMemsetAsync(q, 0, N * sizeof(T), s->st));
    }
    s->nstep = 0;
    CK(cudaMemsetAsync(s->d_status, 0, sizeof(unsigned), s->st));
    CK(cudaMemsetAsync(s->d_maxdiv, 0, sizeof(unsigned long long), s->st));
    CK(cudaStreamSynchronize(s->st));
    return EVP_OK;
}

}  // namespace

extern "C" {

const char* evp_last_error(void) { return g_err.c_str(); }

int evp_num_kernels(void) { return K_COUNT; }

const char* evp_kernel_name(int i) { return (i >= 0 && i < K_COUNT) ? KERNEL_NAMES[i] : ""; }

size_t evp_state_bytes(const evp_grid* grid, evp_model model, const evp_params* params) {
    if (validate(grid, model, params) != EVP_OK) return 0;
    evp_state tmp;
    tmp.g = *grid;
    tmp.model = model;
    tmp.prm = *params;
    tmp.elt = params->precision == EVP_FP32 ? 4 : 8;
    return plan(&tmp, nullptr);
}

int evp_init(const evp_grid* grid, evp_model model, const evp_params* params, void* stream, void* arena,
             size_t arena_bytes, evp_state** out) {
    if (!out) return fail(EVP_ERR_ARG, "null output pointer");
    *out = nullptr;
    int r = validate(grid, model, params);
    if (r) return r;
    evp_state* s = new (std::nothrow) evp_state();
    if (!s) return fail(EVP_ERR_OOM, "host allocation failed");
    s->g = *grid;
    s->model = model;
    s->prm = *params;
    s->fp32 = params->precision == EVP_FP32;
    s->elt = s->fp32 ? 4 : 8;
    s->use_graph = false;
    s->pdl = true;
    s->nvtx = false;
    s->batch = nullptr;
    s->batch_st = nullptr;
    s->n_part = s->n_lag = 0;
    s->ibm_iters = 3;
    s->ibm_block = nullptr;
    s->any_free = 0;
    for (auto& gr : s->graphs) gr.valid = false;
    s->N = (size_t)grid->nx * grid->ny * grid->nz;
    s->nxh = grid->nx / 2 + 1;
    s->timing = false;
    for (int k = 0; k < K_COUNT; ++k) {
        s->ms[k] = 0;
        s->launches[k] = 0;
    }
    const double mu0 = 1.0 / params->Re;
    s->mc.model = model;
    s->mc.inv_lam = model == EVP_NEWTONIAN ? 0.0 : 1.0 / params->Wi;
    s->mc.gmod = model == EVP_NEWTONIAN ? 0.0 : (1.0 - params->beta) * mu0 / params->Wi;
    s->mc.tau_y = params->bi_def == 0 ? params->Bi * mu0 : params->Bi;
    s->mc.L2 = params->L2;
    s->mc.a_fene = model == EVP_FENE_P ? params->L2 / (params->L2 - 3.0) : 1.0;
    s->mc.mu_s = params->beta * mu0;
    s->mc.art_diff = model == EVP_NEWTONIAN ? 0.0 : params->art_diff;
    s->mc.set_single();
    if (stream) {
        s->st = static_cast<cudaStream_t>(stream);
        s->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return cuda_fail(e, "cudaStreamCreate");
        }
        s->own_stream = true;
    }
    const size_t need = plan(s, nullptr);
    if (arena) {
        if (arena_bytes < need) {
            if (s->own_stream) cudaStreamDestroy(s->st);
            delete s;
            return fail(EVP_ERR_OOM, "arena smaller than evp_state_bytes()");
        }
        if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) {
            if (s->own_stream) cudaStreamDestroy(s->st);
            delete s;
            return fail(EVP_ERR_ARG, "arena must be 256-byte aligned");
        }
        s->arena = static_cast<char*>(arena);
        s->own_arena = false;
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) {
            if (s->own_stream) cudaStreamDestroy(s->st);
            delete s;
            cudaGetLastError();
            return fail(EVP_ERR_OOM, std::string("cudaMalloc of the state arena failed: ") + cudaGetErrorString(e));
        }
        s->arena = static_cast<char*>(p);
        s->own_arena = true;
    }
    s->arena_bytes = need;
    plan(s, s->arena);
    s->cu = 0;
    s->cb = 0;
    r = s->fp32 ? upload_tables<float>(s) : upload_tables<double>(s);
    if (!r) r = s->fp32 ? init_fields<float>(s) : init_fields<double>(s);
    if (r) {
        std::string keep = g_err;
        evp_destroy(s);
        g_err = keep;
        return r;
    }
    *out = s;
    return EVP_OK;
}

int evp_destroy(evp_state* s) {
    if (!s) return EVP_OK;
    if (s->batch) evp_batch_evict(static_cast<evp_batch*>(s->batch), s);
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->ibm_block) cudaFree(s->ibm_block);
    for (auto& p : s->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : s->ev_free) cudaEventDestroy(e);
    for (auto& gr : s->graphs)
        if (gr.valid) cudaGraphExecDestroy(gr.exec);
    if (s->own_arena && s->arena) cudaFree(s->arena);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
    return EVP_OK;
}

namespace {
// enqueue the copy of one field into the state on stream st (no synchronisation)
int put_field(evp_state* s, int field, const void* src, int src_on_device, cudaStream_t st) {
    void* dst = field_ptr(s, field);
    const size_t bytes = s->N * s->elt;
    CK(cudaMemcpyAsync(dst, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (field == EVP_V && s->g.walls_y) {
        // the stored top face is the wall: v = 0
        const size_t row = (size_t)s->g.nx * s->elt;
        CK(cudaMemset2DAsync(static_cast<char*>(dst) + (size_t)(s->g.ny - 1) * row, (size_t)s->g.ny * row, 0, row,
                             s->g.nz, st));
    }
    return EVP_OK;
}
int take_field(evp_state* s, int field, void* dst, int dst_on_device, cudaStream_t st) {
    CK(cudaMemcpyAsync(dst, field_ptr(s, field), s->N * s->elt,
                       dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return EVP_OK;
}
}  // namespace

namespace {
// a batch member's steps run on the batch's stream: wait for them before touching
// the state from its own stream
int wait_batch(evp_state* s) {
    if (s->batch) CK(cudaStreamSynchronize(s->batch_st));
    return EVP_OK;
}
}  // namespace

int evp_set_field(evp_state* s, int field, const void* src, int src_on_device) {
    if (!s || !src) return fail(EVP_ERR_ARG, "null state or source");
    if (int r = wait_batch(s)) return r;
    if (field == EVP_PSI) return fail(EVP_ERR_ARG, "EVP_PSI is read only");
    if (!field_ptr(s, field)) return fail(EVP_ERR_ARG, "unknown field id");
    if (int r = put_field(s, field, src, src_on_device, s->st)) return r;
    CK(cudaStreamSynchronize(s->st));
    return EVP_OK;
}

int evp_get_field(evp_state* s, int field, void* dst, int dst_on_device) {
    if (!s || !dst) return fail(EVP_ERR_ARG, "null state or destination");
    if (int r = wait_batch(s)) return r;
    if (!field_ptr(s, field)) return fail(EVP_ERR_ARG, "unknown field id");
    if (int r = take_field(s, field, dst, dst_on_device, s->st)) return r;
    CK(cudaStreamSynchronize(s->st));
    return EVP_OK;
}

int evp_set_fields(evp_state* s, int n, const int* fields, const void* const* srcs, int src_on_device) {
    if (!s || n < 0 || (n > 0 && (!fields || !srcs))) return fail(EVP_ERR_ARG, "null state or arrays, or n < 0");
    if (int r = wait_batch(s)) return r;
    for (int i = 0; i < n; ++i) {
        if (!srcs[i]) return fail(EVP_ERR_ARG, "null source buffer");
        if (fields[i] == EVP_PSI) return fail(EVP_ERR_ARG, "EVP_PSI is read only");
        if (!field_ptr(s, fields[i])) return fail(EVP_ERR_ARG, "unknown field id");
    }
    for (int i = 0; i < n; ++i)
        if (int r = put_field(s, fields[i], srcs[i], src_on_device, s->st)) return r;
    CK(cudaStreamSynchronize(s->st));
    return EVP_OK;
}

int evp_get_fields(evp_state* s, int n, const int* fields, void* const* dsts, int dst_on_device) {
    if (!s || n < 0 || (n > 0 && (!fields || !dsts))) return fail(EVP_ERR_ARG, "null state or arrays, or n < 0");
    if (int r = wait_batch(s)) return r;
    for (int i = 0; i < n; ++i) {
        if (!dsts[i]) return fail(EVP_ERR_ARG, "null destination buffer");
        if (!field_ptr(s, fields[i])) return fail(EVP_ERR_ARG, "unknown field id");
    }
    for (int i = 0; i < n; ++i)
        if (int r = take_field(s, fields[i], dsts[i], dst_on_device, s->st)) return r;
    CK(cudaStreamSynchronize(s->st));
    return EVP_OK;
}

int evp_substep(evp_state* s, double dt, int k) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    if (s->batch) return fail(EVP_ERR_STATE, "the state is a member of a batch: it steps with evp_batch_step");
    if (s->ab2) return fail(EVP_ERR_STATE, "evp_substep is an RK3 call; this state integrates with AB2");
    if (k < 0 || k > 2) return fail(EVP_ERR_ARG, "substep index must be 0, 1 or 2");
    if (!(dt > 0)) return fail(EVP_ERR_ARG, "dt must be positive");
    if (int r = prepare_helmholtz(s, dt)) return r;
    static const char* const SUBSTEP_NAMES[3] = {"evp_substep 0", "evp_substep 1", "evp_substep 2"};
    NvtxScope range(s, SUBSTEP_NAMES[k]);
    return s->fp32 ? substep_t<float>(s, dt, k, false) : substep_t<double>(s, dt, k, false);
}

namespace {
int rk3_step_direct(evp_state* s, double dt) {
    for (int k = 0; k < 3; ++k) {
        int r = s->fp32 ? substep_t<float>(s, dt, k, k == 2) : substep_t<double>(s, dt, k, k == 2);
        if (r) return r;
    }
    return EVP_OK;
}

// Replay (capturing on first use) the graph of one RK3 step for this dt and B parity.
int rk3_step_graph(evp_state* s, double dt) {
    auto& gr = s->graphs[s->cb];
    if (!gr.valid || gr.dt != dt) {
        if (gr.valid) {
            cudaGraphExecDestroy(gr.exec);
            gr.valid = false;
        }
        const int cu0 = s->cu, cb0 = s->cb;
        cudaError_t eb = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
        int r = EVP_OK;
        cudaGraph_t graph = nullptr;
        cudaError_t ec = eb;
        if (eb == cudaSuccess) {
            // graph replay already hides launch latency; programmatic dependent
            // launch inside the graph measured slower (1.74 vs 1.72 ms per channel
            // step), so the graph's kernels are captured as plain launches
            const bool pdl0 = s->pdl;
            s->pdl = false;
            r = rk3_step_direct(s, dt);
            s->pdl = pdl0;
            ec = cudaStreamEndCapture(s->st, &graph);
        }
        const int cb_after = s->cb;
        s->cu = cu0;
        s->cb = cb0;
        cudaError_t ei = cudaErrorUnknown;
        if (r == EVP_OK && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&gr.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            // capture is not available on this stream: run the step directly from now on
            cudaGetLastError();
            s->use_graph = false;
            return rk3_step_direct(s, dt);
        }
        gr.valid = true;
        gr.dt = dt;
        gr.cb_after = cb_after;
    }
    CK(cudaGraphLaunch(gr.exec, s->st));
    s->cb = gr.cb_after;
    return EVP_OK;
}
}  // namespace

extern "C" int evp_set_graph(evp_state* s, int enable) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    if (enable && s->ab2) return fail(EVP_ERR_STATE, "graph replay covers the RK3 step only");
    s->use_graph = enable != 0;
    return EVP_OK;
}

extern "C" int evp_set_nvtx(evp_state* s, int enable) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    s->nvtx = enable != 0;
    return EVP_OK;
}

extern "C" int evp_set_pdl(evp_state* s, int enable) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    CK(cudaStreamSynchronize(s->st));
    s->pdl = enable != 0;
    // captured graphs hold the old launch attributes: capture again on the next step
    for (auto& gr : s->graphs)
        if (gr.valid) {
            cudaGraphExecDestroy(gr.exec);
            gr.valid = false;
        }
    return EVP_OK;
}

extern "C" int evp_set_particles(evp_state* s, int n, const double* desc, int iters) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    if (s->ab2) return fail(EVP_ERR_STATE, "rigid particles belong to the RK3 step");
    if (n < 0 || n > 4096 || (n > 0 && !desc)) return fail(EVP_ERR_ARG, "bad particle count or descriptor");
    if (iters < 1 || iters > 20) return fail(EVP_ERR_ARG, "iters must be 1..20");
    const evp_grid& g = s->g;
    const double dx = g.lx / g.nx, dy = g.ly / g.ny, dz = g.lz / g.nz;
    if (n > 0 && (std::fabs(dx - dy) > 1e-12 * dx || std::fabs(dx - dz) > 1e-12 * dx))
        return fail(EVP_ERR_ARG, "the IBM needs cubic cells (dx = dy = dz)");
    // Lagrangian points (Reading 19): retracted sphere, spiral lattice, equal shell volumes
    std::vector<double> off, dvl, centre, vel, omg, rad, dens;
    std::vector<int> owner, start(1, 0);
    const double golden = M_PI * (3.0 - std::sqrt(5.0));
    for (int p = 0; p < n; ++p) {
        const double* d = desc + 11 * p;
        const double R = d[3];
        if (!(R >= 2.0 * dx)) return fail(EVP_ERR_ARG, "particle radius must be at least 2 dx");
        if (g.walls_y && !(std::fabs(d[1]) + R + 2.0 * dy <= 0.5 * g.ly))
            return fail(EVP_ERR_ARG, "particles must stay R + 2 dy away from the walls");
        for (int q = 0; q < 11; ++q)
            if (!std::isfinite(d[q])) return fail(EVP_ERR_ARG, "non-finite particle descriptor");
        if (d[10] < 0.0) return fail(EVP_ERR_ARG, "particle density ratio must be >= 0 (0: prescribed motion)");
        if (2.0 * (R + 2.0 * dx) >= std::min(g.lx, g.lz) || (!g.walls_y && 2.0 * (R + 2.0 * dy) >= g.ly))
            return fail(EVP_ERR_ARG, "particle too large for the periodic box");
        const double rr = R - 0.3 * dx;
        const int nl = (int)std::lround(M_PI / 3.0 * (12.0 * (rr / dx) * (rr / dx) + 1.0));
        for (int l = 0; l < nl; ++l) {
            const double z = 1.0 - (2.0 * l + 1.0) / nl, rho = std::sqrt(1.0 - z * z), th = golden * l;
            off.push_back(rr * rho * std::cos(th));
            off.push_back(rr * rho * std::sin(th));
            off.push_back(rr * z);
            owner.push_back(p);
        }
        start.push_back(start.back() + nl);
        dvl.push_back(M_PI * dx * (12.0 * rr * rr + dx * dx) / (3.0 * nl));
        for (int q = 0; q < 3; ++q) {
            centre.push_back(d[q]);
            vel.push_back(d[4 + q]);
            omg.push_back(d[7 + q]);
        }
        rad.push_back(R);
        dens.push_back(d[10]);
    }
    CK(cudaStreamSynchronize(s->st));
    for (auto& gr : s->graphs)   // the step graph holds the particle arrays
        if (gr.valid) {
            cudaGraphExecDestroy(gr.exec);
            gr.valid = false;
        }
    if (s->ibm_block) {
        cudaFree(s->ibm_block);
        s->ibm_block = nullptr;
    }
    s->n_part = s->n_lag = 0;
    if (n == 0) return EVP_OK;
    const size_t nl = owner.size();
    const size_t doubles = 3 * nl + n + 3 * n * 3 + 3 * nl * 2 + 6 * n + 2 * n + 12 * n;
    const size_t bytes = doubles * sizeof(double) + (nl + n + 1) * sizeof(int);
    if (cudaMalloc(&s->ibm_block, bytes) != cudaSuccess) {
        cudaGetLastError();
        s->ibm_block = nullptr;
        return fail(EVP_ERR_OOM, "particle arrays");
    }
    double* b = static_cast<double*>(s->ibm_block);
    s->i_off = b;
    s->i_dvl = s->i_off + 3 * nl;
    s->i_centre = s->i_dvl + n;
    s->i_vel = s->i_centre + 3 * n;
    s->i_omg = s->i_vel + 3 * n;
    s->i_Facc = s->i_omg + 3 * n;
    s->i_dF = s->i_Facc + 3 * nl;
    s->i_force = s->i_dF + 3 * nl;
    s->i_rad = s->i_force + 6 * n;
    s->i_dens = s->i_rad + n;
    s->i_int = s->i_dens + n;
    s->i_owner = reinterpret_cast<int*>(s->i_int + 12 * n);
    s->i_start = s->i_owner + nl;
    CK(cudaMemcpy(s->i_off, off.data(), off.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->i_dvl, dvl.data(), dvl.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->i_centre, centre.data(), centre.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->i_vel, vel.data(), vel.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->i_omg, omg.data(), omg.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(s->i_Facc, 0, 3 * nl * sizeof(double)));
    CK(cudaMemset(s->i_force, 0, 6 * n * sizeof(double)));
    CK(cudaMemcpy(s->i_rad, rad.data(), rad.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->i_dens, dens.data(), dens.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(s->i_int, 0, 12 * n * sizeof(double)));
    CK(cudaMemcpy(s->i_owner, owner.data(), owner.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->i_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
    s->n_part = n;
    s->n_lag = (int)nl;
    s->ibm_iters = iters;
    s->any_free = 0;
    for (double r : dens) s->any_free |= r > 0.0;
    return EVP_OK;
}

extern "C" int evp_get_particles(evp_state* s, int n, double* out) {
    if (!s || !out) return fail(EVP_ERR_ARG, "null state or output");
    if (n != s->n_part) return fail(EVP_ERR_ARG, "n must equal the number of particles set");
    if (n == 0) return EVP_OK;
    CK(cudaStreamSynchronize(s->st));
    std::vector<double> c(3 * (size_t)n), u(3 * (size_t)n), w(3 * (size_t)n), f(6 * (size_t)n);
    CK(cudaMemcpy(c.data(), s->i_centre, c.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(u.data(), s->i_vel, u.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(w.data(), s->i_omg, w.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(f.data(), s->i_force, f.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int p = 0; p < n; ++p) {
        for (int q = 0; q < 3; ++q) {
            out[15 * p + q] = c[3 * p + q];
            out[15 * p + 3 + q] = u[3 * p + q];
            out[15 * p + 6 + q] = w[3 * p + q];
        }
        for (int q = 0; q < 6; ++q) out[15 * p + 9 + q] = f[6 * p + q];
    }
    return EVP_OK;
}

extern "C" int evp_step(evp_state* s, double dt) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    if (s->batch) return fail(EVP_ERR_STATE, "the state is a member of a batch: it steps with evp_batch_step");
    if (!(dt > 0)) return fail(EVP_ERR_ARG, "dt must be positive");
    if (int r = prepare_helmholtz(s, dt)) return r;
    if (s->ab2) {
        NvtxScope range(s, "evp_step");
        return s->fp32 ? ab2_step_t<float>(s, dt) : ab2_step_t<double>(s, dt);
    }
    if (s->use_graph && !s->timing) {
        NvtxScope range(s, "evp_step graph replay");
        return rk3_step_graph(s, dt);
    }
    NvtxScope range(s, "evp_step");
    static const char* const SUBSTEP_NAMES[3] = {"evp_substep 0", "evp_substep 1", "evp_substep 2"};
    for (int k = 0; k < 3; ++k) {
        NvtxScope sub(s, SUBSTEP_NAMES[k]);
        int r = s->fp32 ? substep_t<float>(s, dt, k, k == 2) : substep_t<double>(s, dt, k, k == 2);
        if (r) return r;
    }
    return EVP_OK;
}

int evp_step_io(evp_state* s, double dt, int n_in, const int* in_fields, const void* const* in_srcs, int n_out,
                const int* out_fields, void* const* out_dsts) {
    if (!s || n_in < 0 || n_out < 0 || (n_in > 0 && (!in_fields || !in_srcs)) ||
        (n_out > 0 && (!out_fields || !out_dsts)))
        return fail(EVP_ERR_ARG, "null state or arrays, or a negative count");
    if (!(dt > 0)) return fail(EVP_ERR_ARG, "dt must be positive");
    for (int i = 0; i < n_in; ++i) {
        if (!in_srcs[i]) return fail(EVP_ERR_ARG, "null source buffer");
        if (in_fields[i] == EVP_PSI) return fail(EVP_ERR_ARG, "EVP_PSI is read only");
        if (!field_ptr(s, in_fields[i])) return fail(EVP_ERR_ARG, "unknown field id");
    }
    for (int i = 0; i < n_out; ++i) {
        if (!out_dsts[i]) return fail(EVP_ERR_ARG, "null destination buffer");
        if (!field_ptr(s, out_fields[i])) return fail(EVP_ERR_ARG, "unknown field id");
    }
    if (s->batch) return fail(EVP_ERR_STATE, "the state is a member of a batch: it steps with evp_batch_step");
    for (int i = 0; i < n_in; ++i)
        if (int r = put_field(s, in_fields[i], in_srcs[i], 0, s->st)) return r;
    if (int r = evp_step(s, dt)) return r;
    for (int i = 0; i < n_out; ++i)
        if (int r = take_field(s, out_fields[i], out_dsts[i], 0, s->st)) return r;
    return EVP_OK;
}

int evp_project(evp_state* s) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    if (int r = wait_batch(s)) return r;
    const int cu = s->cu;
    int r;
    if (s->fp32) {
        r = run_poisson<float>(s, (const float*)s->U[cu], (const float*)s->V[cu], (const float*)s->W[cu], nullptr,
                               1.0, (float*)s->PSI);
        if (!r)
            r = run_correct<float>(s, (const float*)s->U[cu], (const float*)s->V[cu], (const float*)s->W[cu],
                                   (float*)s->U[1 - cu], (float*)s->V[1 - cu], (float*)s->W[1 - cu], nullptr, 1.0);
    } else {
        r = run_poisson<double>(s, (const double*)s->U[cu], (const double*)s->V[cu], (const double*)s->W[cu],
                                nullptr, 1.0, (double*)s->PSI);
        if (!r)
            r = run_correct<double>(s, (const double*)s->U[cu], (const double*)s->V[cu], (const double*)s->W[cu],
                                    (double*)s->U[1 - cu], (double*)s->V[1 - cu], (double*)s->W[1 - cu], nullptr,
                                    1.0);
    }
    if (!r) s->cu = 1 - cu;
    return r;
}

int evp_poisson_solve(evp_state* s, const void* rhs, void* psi) {
    if (!s || !rhs || !psi) return fail(EVP_ERR_ARG, "null argument");
    if (int r = wait_batch(s)) return r;
    if (s->fp32) return run_poisson<float>(s, nullptr, nullptr, nullptr, (const float*)rhs, 1.0, (float*)psi);
    return run_poisson<double>(s, nullptr, nullptr, nullptr, (const double*)rhs, 1.0, (double*)psi);
}

int evp_stress_rhs(evp_state* s, void* rt) {
    if (!s || !rt) return fail(EVP_ERR_ARG, "null argument");
    if (s->model == EVP_NEWTONIAN) return fail(EVP_ERR_STATE, "a Newtonian state has no stress");
    if (int r = wait_batch(s)) return r;
    auto go = [&](auto tag) -> int {
        using T = decltype(tag);
        StressArgs<T> a;
        const int cu = s->cu, cb = s->cb;
        a.U = static_cast<const T*>(s->U[cu]);
        a.V = static_cast<const T*>(s->V[cu]);
        a.W = static_cast<const T*>(s->W[cu]);
        for (int c = 0; c < 6; ++c) {
            a.B[c] = static_cast<const T*>(s->B[cb][c]);
            a.Bn[c] = nullptr;
            a.RT[c] = static_cast<T*>(rt) + (size_t)c * s->N;
        }
        a.dt_zeta = T(0);
        a.dt_xi = T(0);
        a.read_hist = 0;
        a.write_hist = 0;
        a.rhs_only = 1;
        a.status = s->d_status;
        a.H = nullptr;
        a.mu_p1 = a.mu_p2 = T(0);
        cudaError_t e = launch_stress<T>(geo_of<T>(s), s->mc, a, s->st, hook_of(s));
        return e == cudaSuccess ? EVP_OK : cuda_fail(e, "stress kernel");
    };
    return s->fp32 ? go(float(0)) : go(double(0));
}

int evp_sync(evp_state* s, unsigned* bits, double* max_div) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    if (int r = wait_batch(s)) return r;
    if (max_div) {
        // FP64 max |div u| of the current (last projected) velocity
        CK(cudaMemsetAsync(s->d_maxdiv, 0, sizeof(unsigned long long), s->st));
        const int cu = s->cu;
        const double ix = s->g.nx / s->g.lx, iy = s->g.ny / s->g.ly, iz = s->g.nz / s->g.lz;
        const cudaError_t e = s->fp32
            ? launch_div_residual<float>(geo_of<float>(s), (const float*)s->U[cu], (const float*)s->V[cu],
                                         (const float*)s->W[cu], ix, iy, iz, s->d_maxdiv, s->d_status, s->st)
            : launch_div_residual<double>(geo_of<double>(s), (const double*)s->U[cu], (const double*)s->V[cu],
                                          (const double*)s->W[cu], ix, iy, iz, s->d_maxdiv, s->d_status, s->st);
        if (e != cudaSuccess) return cuda_fail(e, "divergence residual");
    }
    CK(cudaStreamSynchronize(s->st));
    unsigned st = 0;
    unsigned long long md = 0;
    CK(cudaMemcpy(&st, s->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&md, s->d_maxdiv, sizeof(md), cudaMemcpyDeviceToHost));
    CK(cudaMemsetAsync(s->d_status, 0, sizeof(unsigned), s->st));
    CK(cudaStreamSynchronize(s->st));
    if (bits) *bits = st;
    if (max_div) {
        double d;
        std::memcpy(&d, &md, sizeof(d));
        *max_div = d;
    }
    if (st & EVP_BIT_BOUNDS) return fail(EVP_ERR_BOUNDS, "a checked kernel access failed (debug build)");
    if (st & EVP_BIT_NONFINITE) return fail(EVP_ERR_NONFINITE, "non-finite values in the fields");
    if (st & EVP_BIT_TRACE_LIMIT) return fail(EVP_ERR_UNPHYSICAL, "B reached the FENE-P trace limit");
    // with the local artificial diffusion on, det B < 0 is the condition it treats
    if ((st & EVP_BIT_DET_NEG) && !(s->mc.art_diff > 0))
        return fail(EVP_ERR_UNPHYSICAL, "B lost positive definiteness");
    return EVP_OK;
}

int evp_diagnostics(evp_state* s, evp_diag* out) {
    if (!s || !out) return fail(EVP_ERR_ARG, "null state or output");
    if (int r = wait_batch(s)) return r;
    CK(cudaMemsetAsync(s->d_maxdiv, 0, sizeof(unsigned long long), s->st));
    const int cu = s->cu, cb = s->cb;
    const double ix = s->g.nx / s->g.lx, iy = s->g.ny / s->g.ly, iz = s->g.nz / s->g.lz;
    DiagPart* parts = static_cast<DiagPart*>(s->diag);
    DiagPart* res = parts + DIAG_BLOCKS;
    auto go = [&](auto zero) -> int {
        using T = decltype(zero);
        DiagArgs<T> a;
        a.U = static_cast<const T*>(s->U[cu]);
        a.V = static_cast<const T*>(s->V[cu]);
        a.W = static_cast<const T*>(s->W[cu]);
        const bool hasB = s->model != EVP_NEWTONIAN;
        for (int c = 0; c < 6; ++c) a.B[c] = hasB ? static_cast<const T*>(s->B[cb][c]) : nullptr;
        a.H = nullptr;
        a.gm = s->mc.gmod;
        a.mp1 = 0.0;
        a.inv_lam = s->mc.inv_lam;
        a.tau_y = s->mc.tau_y;
        a.yield_mode = (s->model == EVP_OLDROYD_B || s->model == EVP_FENE_P) ? 1
                     : s->model == EVP_SARAMITO ? 2 : 0;
        if (s->ab2 && s->model == EVP_SARAMITO) {
            a.H = static_cast<const T*>(s->HF);
            a.mp1 = (1.0 - s->prm.beta) * (1.0 / s->prm.Re);   // mu_p of fluid 1, as the AB2 step forms it
        }
        cudaError_t e = launch_div_residual<T>(geo_of<T>(s), a.U, a.V, a.W, ix, iy, iz, s->d_maxdiv,
                                               s->d_status, s->st);
        if (e == cudaSuccess) e = launch_diag<T>(geo_of<T>(s), a, parts, res, s->st);
        return e == cudaSuccess ? EVP_OK : cuda_fail(e, "diagnostics kernels");
    };
    // the residual kernel would OR EVP_BIT_NONFINITE into the status word: read the
    // word first and put it back, so that evp_sync reports only what the steps raised
    unsigned st_before = 0;
    CK(cudaMemcpyAsync(&st_before, s->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st));
    if (int r = s->fp32 ? go(float(0)) : go(double(0))) return r;
    DiagPart h;
    unsigned long long md = 0;
    CK(cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(&md, s->d_maxdiv, sizeof(md), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    CK(cudaMemcpyAsync(s->d_status, &st_before, sizeof(unsigned), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    const double dv = s->g.lx / s->g.nx * (s->g.ly / s->g.ny) * (s->g.lz / s->g.nz);
    out->kinetic_energy = 0.5 * dv * h.ke;
    std::memcpy(&out->max_div, &md, sizeof(double));
    const bool hasB = s->model != EVP_NEWTONIAN;
    out->min_det_B = hasB ? h.min_det : std::numeric_limits<double>::infinity();
    out->max_tr_B = hasB ? h.max_tr : 0.0;
    out->max_tr_B_over_L2 = s->model == EVP_FENE_P ? h.max_tr / s->prm.L2 : 0.0;
    out->yielded_cells = h.yielded;
    out->yielded_fraction = double(h.yielded) / double(s->N);
    out->nonfinite_cells = h.nonfinite;
    return EVP_OK;
}

int evp_selftest(unsigned long long* mismatches) {
    if (!mismatches) return fail(EVP_ERR_ARG, "null output");
    const cudaError_t e = evp::run_selftest(mismatches);
    if (e != cudaSuccess) return cuda_fail(e, "self-test kernels");
    return EVP_OK;
}

int evp_fma_peak(int precision, double* flops_per_s) {
    if (!flops_per_s) return fail(EVP_ERR_ARG, "null output");
    if (precision != EVP_FP64 && precision != EVP_FP32) return fail(EVP_ERR_ARG, "bad precision");
    const cudaError_t e = evp::run_fma_peak(precision, flops_per_s);
    if (e != cudaSuccess) return cuda_fail(e, "peak kernels");
    return EVP_OK;
}

int evp_kernel_timing(evp_state* s, int enable) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    flush_timing(s);
    s->timing = enable != 0;
    return EVP_OK;
}

int evp_kernel_times(evp_state* s, double* ms, long long* launches, int n) {
    if (!s) return fail(EVP_ERR_ARG, "null state");
    flush_timing(s);
    for (int k = 0; k < n && k < K_COUNT; ++k) {
        if (ms) ms[k] = s->ms[k];
        if (launches) launches[k] = s->launches[k];
    }
    for (int k = 0; k < K_COUNT; ++k) {
        s->ms[k] = 0;
        s->launches[k] = 0;
    }
    return EVP_OK;
}

}  // extern "C"
