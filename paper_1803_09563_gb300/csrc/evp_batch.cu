// Batched RK3 steps of many simulations (evp_batch_* of evp.h) and the tile
// autotuner (evp_tune).  The paper runs one simulation per job; serving many at
// once is this library's own addition.
//
// One evp_batch_step advances every member by one RK3 step (Eq. RK) of its own dt
// with one launch per kernel phase and substep:
//   * stress update (S1 + S2) and momentum predictor (S3): persistent kernels over a
//     device work list of (member, tile x, tile y, z chunk), members of any grid;
//   * Poisson passes (S4 - S7) and correction (S8): one launch per pass for each
//     group of members on the same grid, the member in blockIdx.z.
// Members' argument blocks travel in the kernels' parameter space.  Each member's
// arithmetic is that of its own evp_step, cell for cell, so results agree bit for
// bit with the member stepped alone.  Steps are captured into CUDA graphs, one per
// (membership, dts, buffer parities), and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "evp_internal.cuh"
#include "evp_state.cuh"

using namespace evp;

// The members' argument blocks travel in the batched kernels' parameter space
// (at most 32764 bytes with the work-list pointer and count).
static_assert(sizeof(MomentumBatch<double>) + 16 <= 32764, "momentum batch parameters too large");
static_assert(sizeof(StressBatch<double>) + 16 <= 32764, "stress batch parameters too large");

namespace {

int bfail(int code, const std::string& m) {
    set_last_error(m);
    return code;
}
int bcuda(cudaError_t e, const char* where) {
    set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
    return EVP_ERR_CUDA;
}
#define BCK(call)                                               \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return bcuda(e_, #call);         \
    } while (0)

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// ------------------------------------------------------------ tile configs
using CfgKey = std::tuple<int, int, int, int, int, int>;   // nx, ny, nz, walls, precision, model
std::mutex g_cfg_mutex;
std::map<CfgKey, evp_tile_config> g_cfg;

CfgKey cfg_key(const evp_grid& g, int precision, int model) {
    return CfgKey(g.nx, g.ny, g.nz, g.walls_y ? 1 : 0, precision, model);
}

// z planes per work item of the single-state launches: about four waves of CTAs
int default_kz(int nx, int ny, int nz, int tx, int ty, int per_sm) {
    const int tiles = ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
    int chunks = (4 * 152 * per_sm + tiles - 1) / tiles;
    chunks = chunks > nz ? nz : chunks;
    return (nz + chunks - 1) / chunks;
}

evp_tile_config default_config(const evp_grid& g, int precision) {
    const bool f32 = precision == EVP_FP32;
    evp_tile_config c;
    c.stress_ctas_per_sm = f32 ? stress_ctas_per_sm<float>() : stress_ctas_per_sm<double>();
    c.momentum_ctas_per_sm = f32 ? momentum_ctas_per_sm<float>() : momentum_ctas_per_sm<double>();
    c.stress_kz = default_kz(g.nx, g.ny, g.nz, stress_tile_x(), stress_tile_y(), c.stress_ctas_per_sm);
    c.momentum_kz = default_kz(g.nx, g.ny, g.nz, momentum_tile_x(), momentum_tile_y(), c.momentum_ctas_per_sm);
    c.fft_cols = f32 ? 16 : 8;
    return c;
}

// fill zero fields with the defaults; false if a field is out of range
bool complete_config(const evp_grid& g, int precision, evp_tile_config& c) {
    const evp_tile_config d = default_config(g, precision);
    if (!c.stress_kz) c.stress_kz = d.stress_kz;
    if (!c.momentum_kz) c.momentum_kz = d.momentum_kz;
    if (!c.stress_ctas_per_sm) c.stress_ctas_per_sm = d.stress_ctas_per_sm;
    if (!c.momentum_ctas_per_sm) c.momentum_ctas_per_sm = d.momentum_ctas_per_sm;
    if (!c.fft_cols) c.fft_cols = d.fft_cols;
    const bool f32 = precision == EVP_FP32;
    return c.stress_kz >= 1 && c.stress_kz <= g.nz && c.momentum_kz >= 1 && c.momentum_kz <= g.nz &&
           c.stress_ctas_per_sm >= 1 && c.stress_ctas_per_sm <= d.stress_ctas_per_sm && c.momentum_ctas_per_sm >= 1 &&
           c.momentum_ctas_per_sm <= d.momentum_ctas_per_sm &&
           (c.fft_cols == 4 || c.fft_cols == 8 || (c.fft_cols == 16 && f32));
}

evp_tile_config lookup_config(const evp_grid& g, int precision, int model) {
    {
        std::lock_guard<std::mutex> lock(g_cfg_mutex);
        auto it = g_cfg.find(cfg_key(g, precision, model));
        if (it != g_cfg.end()) return it->second;
    }
    return default_config(g, precision);
}

bool same_grid(const evp_grid& a, const evp_grid& b) {
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.lx == b.lx && a.ly == b.ly && a.lz == b.lz &&
           a.walls_y == b.walls_y;
}

}  // namespace

struct evp_batch_s {
    int precision = EVP_FP32;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    struct Member {
        evp_state* s;
        double dt;
        evp_tile_config cfg;
    };
    std::vector<Member> m;
    bool use_graph = true;
    bool dirty = true;          // membership changed: launch plan and graphs are stale
    bool has_override = false;  // the tuner's trial configuration for every member
    evp_tile_config override_cfg{};
    // launch plan: the persistent launches and the same-grid groups
    struct Launch {
        std::vector<int> idx;   // members, in parameter-array order
        int model = 0;
        bool vec = true;
        int work_off = 0, nwork = 0, ctas = 0;
    };
    std::vector<Launch> stress, momentum;
    struct Group {
        std::vector<int> idx;
        int tk = 16;
    };
    std::vector<Group> groups;
    int4* d_work = nullptr;
    size_t work_cap = 0;
    // replayed steps: one executable graph per signature (cu, cb, dt of every member)
    struct Graph {
        bool valid = false;
        std::vector<long long> sig;
        std::vector<int> cb_after;
        cudaGraphExec_t exec = nullptr;
    } graphs[2];
    int next_graph = 0;
};

namespace {

void drop_graphs(evp_batch* b) {
    for (auto& g : b->graphs) {
        if (g.valid) cudaGraphExecDestroy(g.exec);
        g.valid = false;
        g.sig.clear();
    }
}

bool has_vec(const evp_state* s) { return ((size_t)s->g.nx * s->elt) % 16 == 0; }

// Work list entries (member index within its launch, tile x, tile y, z chunk) of
// a z-marching kernel with tx x ty tiles and kz planes per item.
void add_work(std::vector<int4>& w, int gi, const evp_grid& g, int tx, int ty, int kz) {
    const int nbx = (g.nx + tx - 1) / tx, nby = (g.ny + ty - 1) / ty, nbz = (g.nz + kz - 1) / kz;
    for (int bz = 0; bz < nbz; ++bz)
        for (int by = 0; by < nby; ++by)
            for (int bx = 0; bx < nbx; ++bx) w.push_back(make_int4(gi, bx, by, bz));
}

// Rebuild the launch plan after a membership change: configurations, groups and
// the device work lists (the batch's stream is idle when this writes them).
int prepare(evp_batch* b) {
    if (!b->dirty) return EVP_OK;
    BCK(cudaStreamSynchronize(b->st));
    drop_graphs(b);
    b->stress.clear();
    b->momentum.clear();
    b->groups.clear();
    for (auto& mb : b->m)
        mb.cfg = b->has_override ? b->override_cfg : lookup_config(mb.s->g, b->precision, mb.s->model);
    for (int i = 0; i < (int)b->m.size(); ++i) {
        const evp_state* s = b->m[i].s;
        const bool v = has_vec(s);
        auto put = [&](std::vector<evp_batch_s::Launch>& L, int model) {
            for (auto& l : L)
                if (l.model == model && l.vec == v) {
                    l.idx.push_back(i);
                    return;
                }
            evp_batch_s::Launch l;
            l.model = model;
            l.vec = v;
            l.idx.push_back(i);
            L.push_back(l);
        };
        put(b->stress, s->model);
        put(b->momentum, 0);
        bool placed = false;
        for (auto& gr : b->groups)
            if (same_grid(b->m[gr.idx[0]].s->g, s->g) &&
                b->m[gr.idx[0]].s->prm.thomas_fp64 == s->prm.thomas_fp64) {   // same Thomas tables
                gr.idx.push_back(i);
                placed = true;
                break;
            }
        if (!placed) {
            evp_batch_s::Group gr;
            gr.idx.push_back(i);
            gr.tk = b->m[i].cfg.fft_cols;
            b->groups.push_back(gr);
        }
    }
    std::vector<int4> work;
    const int sms = num_sms();
    for (auto& l : b->stress) {
        l.work_off = (int)work.size();
        int per_sm = 1;
        for (int gi = 0; gi < (int)l.idx.size(); ++gi) {
            const auto& mb = b->m[l.idx[gi]];
            add_work(work, gi, mb.s->g, stress_tile_x(), stress_tile_y(), mb.cfg.stress_kz);
            per_sm = std::max(per_sm, mb.cfg.stress_ctas_per_sm);
        }
        l.nwork = (int)work.size() - l.work_off;
        l.ctas = per_sm * sms;
    }
    for (auto& l : b->momentum) {
        l.work_off = (int)work.size();
        int per_sm = 1;
        for (int gi = 0; gi < (int)l.idx.size(); ++gi) {
            const auto& mb = b->m[l.idx[gi]];
            add_work(work, gi, mb.s->g, momentum_tile_x(), momentum_tile_y(), mb.cfg.momentum_kz);
            per_sm = std::max(per_sm, mb.cfg.momentum_ctas_per_sm);
        }
        l.nwork = (int)work.size() - l.work_off;
        l.ctas = per_sm * sms;
    }
    if (work.size() > b->work_cap) {
        if (b->d_work) cudaFree(b->d_work);
        b->d_work = nullptr;
        b->work_cap = 0;
        const size_t cap = std::max<size_t>(work.size(), 4096);
        if (cudaMalloc(&b->d_work, cap * sizeof(int4)) != cudaSuccess) {
            cudaGetLastError();
            return bfail(EVP_ERR_OOM, "device allocation of the batch work list failed");
        }
        b->work_cap = cap;
    }
    if (!work.empty()) BCK(cudaMemcpy(b->d_work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->dirty = false;
    return EVP_OK;
}

}  // namespace

namespace {

// One RK3 step of every member with direct launches (also what a graph captures).
template <typename T>
int step_direct(evp_batch* b) {
    std::unique_ptr<StressBatch<T>> sp(new (std::nothrow) StressBatch<T>());
    std::unique_ptr<MomentumBatch<T>> mp(new (std::nothrow) MomentumBatch<T>());
    std::unique_ptr<PoissonBatch<T>> pp(new (std::nothrow) PoissonBatch<T>());
    std::unique_ptr<CorrectBatch<T>> cp(new (std::nothrow) CorrectBatch<T>());
    if (!sp || !mp || !pp || !cp) return bfail(EVP_ERR_OOM, "host allocation of the batch arguments failed");
    for (int k = 0; k < 3; ++k) {
        const double al = RK_ALPHA[k], ze = RK_ZETA[k], xi = RK_XI[k];
        const bool read_hist = xi != 0.0, write_hist = k != 2;
        const int mode = !read_hist ? 1 : (write_hist ? 2 : 3);
        // ---- S1 + S2: stress update (Eq. rk3tau), one persistent launch per (model, staging)
        for (const auto& l : b->stress) {
            for (int gi = 0; gi < (int)l.idx.size(); ++gi) {
                const auto& mb = b->m[l.idx[gi]];
                evp_state* s = mb.s;
                const double dt = mb.dt;
                StressMember<T>& M = sp->m[gi];
                M.g = geo_of<T>(s);
                M.mc = s->mc;
                M.kz = mb.cfg.stress_kz;
                StressArgs<T>& a = M.a;
                const int cu = s->cu, cb = s->cb;
                a.U = static_cast<const T*>(s->U[cu]);
                a.V = static_cast<const T*>(s->V[cu]);
                a.W = static_cast<const T*>(s->W[cu]);
                for (int c = 0; c < 6; ++c) {
                    a.B[c] = static_cast<const T*>(s->B[cb][c]);
                    a.Bn[c] = static_cast<T*>(s->B[1 - cb][c]);
                    a.RT[c] = static_cast<T*>(s->RT[c]);
                    a.S[c] = static_cast<T*>(s->S[c]);
                }
                a.dt_zeta = T(dt * ze);
                a.dt_xi = T(dt * xi);
                a.read_hist = read_hist;
                a.write_hist = write_hist;
                a.rhs_only = 0;
                a.status = s->d_status;
                a.H = nullptr;
                a.mu_p1 = a.mu_p2 = T(0);
            }
            const cudaError_t e =
                launch_stress_batch<T>(*sp, l.model, mode, l.vec, b->d_work + l.work_off, l.nwork, l.ctas, b->st);
            if (e != cudaSuccess) return bcuda(e, "batched stress kernel");
        }
        // ---- S3: momentum predictor (Eq. rk3) with the summed stress
        for (const auto& l : b->momentum) {
            for (int gi = 0; gi < (int)l.idx.size(); ++gi) {
                const auto& mb = b->m[l.idx[gi]];
                evp_state* s = mb.s;
                const double dt = mb.dt;
                MomentumMember<T>& M = mp->m[gi];
                M.g = geo_of<T>(s);
                M.mc = s->mc;
                M.kz = mb.cfg.momentum_kz;
                MomentumArgs<T>& a = M.a;
                a = MomentumArgs<T>();
                a.status = s->d_status;
                const int cu = s->cu, cb = s->cb;
                a.U = static_cast<const T*>(s->U[cu]);
                a.V = static_cast<const T*>(s->V[cu]);
                a.W = static_cast<const T*>(s->W[cu]);
                a.P = static_cast<const T*>(s->P);
                for (int c = 0; c < 6; ++c) {
                    a.Bo[c] = static_cast<const T*>(s->B[cb][c]);
                    a.Bn[c] = static_cast<const T*>(s->B[1 - cb][c]);
                    a.S[c] = static_cast<const T*>(s->S[c]);
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
                a.has_stress = 1;
                a.dpdx = T(s->prm.dpdx);
                a.abc_amp = T(s->prm.abc_amp);
                a.trig = s->prm.abc_amp != 0.0 ? static_cast<const T*>(s->trig) : nullptr;
                for (int q = 0; q < 3; ++q) a.solid[q] = nullptr;
                a.cn = 0;
            }
            const cudaError_t e =
                launch_momentum_batch<T>(*mp, l.vec, b->d_work + l.work_off, l.nwork, l.ctas, b->st);
            if (e != cudaSuccess) return bcuda(e, "batched momentum kernel");
        }
        // ---- S4 - S8: Poisson passes and correction per same-grid group
        for (const auto& gr : b->groups) {
            const int n = (int)gr.idx.size();
            for (int gi = 0; gi < n; ++gi) {
                const auto& mb = b->m[gr.idx[gi]];
                evp_state* s = mb.s;
                const double coef = 2.0 * al * mb.dt;
                const int cu = s->cu;
                PoissonArgs<T>& a = pp->a[gi];
                a = PoissonArgs<T>();
                a.Us = static_cast<const T*>(s->U[1 - cu]);
                a.Vs = static_cast<const T*>(s->V[1 - cu]);
                a.Ws = static_cast<const T*>(s->W[1 - cu]);
                a.rhs = nullptr;
                a.rscale = T(1.0 / coef);
                a.spec = static_cast<typename Cplx<T>::type*>(s->spec);
                a.psi = static_cast<T*>(s->PSI);
                a.norm = poisson_norm<T>(s);
                a.out_scale = s->g.walls_y ? T(a.norm) : T(1);
                a.scratch = s->thomas_d;
                CorrectArgs<T>& c = cp->a[gi];
                c.Us = a.Us;
                c.Vs = a.Vs;
                c.Ws = a.Ws;
                c.psi = a.psi;
                c.U = static_cast<T*>(s->U[cu]);
                c.V = static_cast<T*>(s->V[cu]);
                c.W = static_cast<T*>(s->W[cu]);
                c.P = static_cast<T*>(s->P);
                c.p_replace = 0;
                c.coef = T(coef);
                c.status = s->d_status;
            }
            const evp_state* s0 = b->m[gr.idx[0]].s;
            cudaError_t e = launch_poisson_batch<T>(geo_of<T>(s0), tables_of<T>(s0), *pp, n, gr.tk, b->st);
            if (e != cudaSuccess) return bcuda(e, "batched Poisson passes");
            e = launch_correct_batch<T>(geo_of<T>(s0), *cp, n, b->st);
            if (e != cudaSuccess) return bcuda(e, "batched correction");
        }
        for (auto& mb : b->m) mb.s->cb = 1 - mb.s->cb;
    }
    return EVP_OK;
}

int run_direct(evp_batch* b) { return b->precision == EVP_FP32 ? step_direct<float>(b) : step_direct<double>(b); }

std::vector<long long> signature(const evp_batch* b) {
    std::vector<long long> sig;
    for (const auto& mb : b->m) {
        long long d;
        std::memcpy(&d, &mb.dt, sizeof d);
        sig.push_back(mb.s->cu);
        sig.push_back(mb.s->cb);
        sig.push_back(d);
    }
    return sig;
}

int step_graph(evp_batch* b) {
    const std::vector<long long> sig = signature(b);
    evp_batch_s::Graph* gr = nullptr;
    for (auto& g : b->graphs)
        if (g.valid && g.sig == sig) gr = &g;
    if (!gr) {
        gr = &b->graphs[b->next_graph];
        b->next_graph ^= 1;
        if (gr->valid) cudaGraphExecDestroy(gr->exec);
        gr->valid = false;
        std::vector<int> cb0;
        for (auto& mb : b->m) cb0.push_back(mb.s->cb);
        cudaGraph_t graph = nullptr;
        int r = EVP_OK;
        cudaError_t ec = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (ec == cudaSuccess) {
            r = run_direct(b);
            ec = cudaStreamEndCapture(b->st, &graph);
        }
        gr->cb_after.clear();
        for (size_t i = 0; i < b->m.size(); ++i) {
            gr->cb_after.push_back(b->m[i].s->cb);
            b->m[i].s->cb = cb0[i];
        }
        cudaError_t ei = cudaErrorUnknown;
        if (r == EVP_OK && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&gr->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (r != EVP_OK) return r;
        if (ei != cudaSuccess) {
            // the stream cannot be captured: launch directly from now on
            cudaGetLastError();
            b->use_graph = false;
            return run_direct(b);
        }
        gr->valid = true;
        gr->sig = sig;
    }
    BCK(cudaGraphLaunch(gr->exec, b->st));
    for (size_t i = 0; i < b->m.size(); ++i) b->m[i].s->cb = gr->cb_after[i];
    return EVP_OK;
}

}  // namespace

extern "C" {

int evp_batch_create(int precision, size_t budget_bytes, void* stream, evp_batch** out) {
    if (!out) return bfail(EVP_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (precision != EVP_FP32 && precision != EVP_FP64) return bfail(EVP_ERR_ARG, "bad precision");
    evp_batch* b = new (std::nothrow) evp_batch();
    if (!b) return bfail(EVP_ERR_OOM, "host allocation failed");
    b->precision = precision;
    b->budget = budget_bytes;
    if (stream) {
        b->st = static_cast<cudaStream_t>(stream);
    } else {
        const cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return bcuda(e, "cudaStreamCreate");
        }
        b->own_stream = true;
    }
    *out = b;
    return EVP_OK;
}

int evp_batch_admit(evp_batch* b, evp_state* s, double dt) {
    if (!b || !s) return bfail(EVP_ERR_ARG, "null batch or state");
    if (!(dt > 0)) return bfail(EVP_ERR_ARG, "dt must be positive");
    if (s->batch) return bfail(EVP_ERR_ARG, "the state is already a member of a batch");
    if (s->prm.precision != b->precision) return bfail(EVP_ERR_ARG, "the state's precision differs from the batch's");
    if (s->ab2) return bfail(EVP_ERR_ARG, "batches hold RK3 states only");
    if (s->model != EVP_OLDROYD_B && s->model != EVP_FENE_P && s->model != EVP_SARAMITO)
        return bfail(EVP_ERR_ARG, "batch members need an Oldroyd-B, FENE-P or Saramito stress");
    if (!s->S[0] || s->prm.penalization || s->prm.soft_particles || s->prm.viscous_implicit || s->n_part > 0 ||
        s->mc.art_diff > 0.0)
        return bfail(EVP_ERR_ARG, "batch members take no penalisation, particles, soft particles, implicit viscous "
                                  "option or artificial diffusion");
    if ((int)b->m.size() >= EVP_BATCH_MAX) return bfail(EVP_ERR_OOM, "the batch holds its maximum of 64 members");
    if (b->budget && b->used + s->arena_bytes > b->budget)
        return bfail(EVP_ERR_OOM, "admitting the state would exceed the batch's memory budget");
    BCK(cudaStreamSynchronize(s->st));
    BCK(cudaStreamSynchronize(b->st));
    b->m.push_back({s, dt, evp_tile_config{}});
    b->used += s->arena_bytes;
    s->batch = b;
    s->batch_st = b->st;
    b->dirty = true;
    return EVP_OK;
}

int evp_batch_evict(evp_batch* b, evp_state* s) {
    if (!b || !s) return bfail(EVP_ERR_ARG, "null batch or state");
    auto it = std::find_if(b->m.begin(), b->m.end(), [&](const evp_batch_s::Member& mb) { return mb.s == s; });
    if (it == b->m.end()) return bfail(EVP_ERR_ARG, "the state is not a member of this batch");
    BCK(cudaStreamSynchronize(b->st));
    b->used -= s->arena_bytes;
    b->m.erase(it);
    s->batch = nullptr;
    s->batch_st = nullptr;
    b->dirty = true;
    return EVP_OK;
}

int evp_batch_step(evp_batch* b) {
    if (!b) return bfail(EVP_ERR_ARG, "null batch");
    if (b->m.empty()) return EVP_OK;
    if (int r = prepare(b)) return r;
    return b->use_graph ? step_graph(b) : run_direct(b);
}

int evp_batch_info(const evp_batch* b, int* members, size_t* bytes) {
    if (!b) return bfail(EVP_ERR_ARG, "null batch");
    if (members) *members = (int)b->m.size();
    if (bytes) *bytes = b->used;
    return EVP_OK;
}

int evp_batch_set_graph(evp_batch* b, int enable) {
    if (!b) return bfail(EVP_ERR_ARG, "null batch");
    b->use_graph = enable != 0;
    return EVP_OK;
}

int evp_batch_destroy(evp_batch* b) {
    if (!b) return EVP_OK;
    cudaStreamSynchronize(b->st);
    for (auto& mb : b->m) {
        mb.s->batch = nullptr;
        mb.s->batch_st = nullptr;
    }
    b->m.clear();
    drop_graphs(b);
    if (b->d_work) cudaFree(b->d_work);
    if (b->own_stream) cudaStreamDestroy(b->st);
    delete b;
    return EVP_OK;
}

int evp_tile_config_set(const evp_grid* grid, int precision, evp_model model, const evp_tile_config* cfg) {
    if (!grid || !cfg) return bfail(EVP_ERR_ARG, "null argument");
    if (precision != EVP_FP32 && precision != EVP_FP64) return bfail(EVP_ERR_ARG, "bad precision");
    evp_tile_config c = *cfg;
    std::lock_guard<std::mutex> lock(g_cfg_mutex);
    if (!c.stress_kz && !c.momentum_kz && !c.stress_ctas_per_sm && !c.momentum_ctas_per_sm && !c.fft_cols) {
        g_cfg.erase(cfg_key(*grid, precision, model));
        return EVP_OK;
    }
    if (!complete_config(*grid, precision, c)) return bfail(EVP_ERR_ARG, "tile configuration out of range");
    g_cfg[cfg_key(*grid, precision, model)] = c;
    return EVP_OK;
}

int evp_tile_config_get(const evp_grid* grid, int precision, evp_model model, evp_tile_config* out) {
    if (!grid || !out) return bfail(EVP_ERR_ARG, "null argument");
    if (precision != EVP_FP32 && precision != EVP_FP64) return bfail(EVP_ERR_ARG, "bad precision");
    *out = lookup_config(*grid, precision, model);
    return EVP_OK;
}

}  // extern "C"

namespace {

// Scratch one-member batch for timing trials: a state of the tuned grid with a
// smooth, exactly solenoidal velocity (each component independent of its own
// coordinate), B = I, and a small dt so that the trials stay far from any limit.
struct Scratch {
    evp_state* s = nullptr;
    evp_batch* b = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
        if (b) evp_batch_destroy(b);
        if (s) evp_destroy(s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

template <typename T>
int scratch_velocity(evp_state* s) {
    const evp_grid& g = s->g;
    const double tp = 6.283185307179586476925286766559;
    std::vector<T> u(s->N), v(s->N), w(s->N);
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) {
                const size_t o = ((size_t)k * g.ny + j) * g.nx + i;
                const double x = (i + 0.5) / g.nx, y = (j + 0.5) / g.ny, z = (k + 0.5) / g.nz;
                const double yy = g.walls_y ? 1.0 - (2 * y - 1) * (2 * y - 1) : std::sin(tp * y);
                u[o] = T(0.5 * std::cos(tp * z) * yy);
                v[o] = T(g.walls_y ? 0.0 : 0.3 * std::sin(tp * x) * std::cos(tp * z));
                w[o] = T(0.4 * std::sin(tp * x) * yy);
            }
    if (int r = evp_set_field(s, EVP_U, u.data(), 0)) return r;
    if (int r = evp_set_field(s, EVP_V, v.data(), 0)) return r;
    return evp_set_field(s, EVP_W, w.data(), 0);
}

int make_scratch(const evp_grid* grid, evp_model model, const evp_params* params, Scratch& sc) {
    if (int r = evp_init(grid, model, params, nullptr, nullptr, 0, &sc.s)) return r;
    if (int r = params->precision == EVP_FP32 ? scratch_velocity<float>(sc.s) : scratch_velocity<double>(sc.s))
        return r;
    if (int r = evp_batch_create(params->precision, 0, nullptr, &sc.b)) return r;
    const double h = std::min(grid->lx / grid->nx, std::min(grid->ly / grid->ny, grid->lz / grid->nz));
    if (int r = evp_batch_admit(sc.b, sc.s, 1e-3 * h)) return r;
    sc.b->has_override = true;
    BCK(cudaEventCreate(&sc.e0));
    BCK(cudaEventCreate(&sc.e1));
    return EVP_OK;
}

// median over three runs of `steps` replayed steps, ms per step
int time_config(Scratch& sc, const evp_tile_config& c, int steps, double* ms) {
    sc.b->override_cfg = c;
    sc.b->dirty = true;
    for (int w = 0; w < 2; ++w)
        if (int r = evp_batch_step(sc.b)) return r;
    double t[3];
    for (int rep = 0; rep < 3; ++rep) {
        BCK(cudaEventRecord(sc.e0, sc.b->st));
        for (int q = 0; q < steps; ++q)
            if (int r = evp_batch_step(sc.b)) return r;
        BCK(cudaEventRecord(sc.e1, sc.b->st));
        BCK(cudaEventSynchronize(sc.e1));
        float f = 0.f;
        BCK(cudaEventElapsedTime(&f, sc.e0, sc.e1));
        t[rep] = f / steps;
    }
    std::sort(t, t + 3);
    *ms = t[1];
    return EVP_OK;
}

std::vector<int> kz_candidates(int nz) {
    std::vector<int> v;
    for (int k = 1; k <= nz && k <= 128; k *= 2) v.push_back(k);
    return v;
}

}  // namespace

extern "C" {

int evp_tile_time(const evp_grid* grid, evp_model model, const evp_params* params, const evp_tile_config* cfg,
                  int steps, double* ms_per_step) {
    if (!grid || !params || !cfg || !ms_per_step || steps < 1) return bfail(EVP_ERR_ARG, "bad argument");
    evp_tile_config c = *cfg;
    if (!complete_config(*grid, params->precision, c)) return bfail(EVP_ERR_ARG, "tile configuration out of range");
    Scratch sc;
    if (int r = make_scratch(grid, model, params, sc)) return r;
    return time_config(sc, c, steps, ms_per_step);
}

int evp_tune(const evp_grid* grid, evp_model model, const evp_params* params, int exhaustive, evp_tile_config* best,
             double* best_ms, int* trials) {
    if (!grid || !params) return bfail(EVP_ERR_ARG, "null grid or params");
    Scratch sc;
    if (int r = make_scratch(grid, model, params, sc)) return r;
    const int prec = params->precision;
    const evp_tile_config d = default_config(*grid, prec);
    const std::vector<int> kz = kz_candidates(grid->nz);
    std::vector<int> sc_c, mc_c, fc;
    for (int q = 1; q <= d.stress_ctas_per_sm; ++q) sc_c.push_back(q);
    for (int q = 1; q <= d.momentum_ctas_per_sm; ++q) mc_c.push_back(q);
    fc.push_back(4);
    fc.push_back(8);
    if (prec == EVP_FP32) fc.push_back(16);
    // steps per timed run: about a millisecond of work or more
    const double cells = (double)grid->nx * grid->ny * grid->nz;
    const int steps = std::max(3, std::min(50, (int)(2e6 / cells) + 1));
    std::map<std::tuple<int, int, int, int, int>, double> seen;
    int n_trials = 0;
    auto trial = [&](const evp_tile_config& c, double* ms) -> int {
        const auto key = std::make_tuple(c.stress_kz, c.momentum_kz, c.stress_ctas_per_sm, c.momentum_ctas_per_sm,
                                         c.fft_cols);
        auto it = seen.find(key);
        if (it != seen.end()) {
            *ms = it->second;
            return EVP_OK;
        }
        if (int r = time_config(sc, c, steps, ms)) return r;
        ++n_trials;
        seen[key] = *ms;
        return EVP_OK;
    };
    evp_tile_config cur = d;
    double cur_ms = 0.0;
    if (int r = trial(cur, &cur_ms)) return r;
    if (exhaustive) {
        for (int a : kz)
            for (int bkz : kz)
                for (int c1 : sc_c)
                    for (int c2 : mc_c)
                        for (int f : fc) {
                            evp_tile_config c{a, bkz, c1, c2, f};
                            double ms = 0.0;
                            if (int r = trial(c, &ms)) return r;
                            if (ms < cur_ms) {
                                cur = c;
                                cur_ms = ms;
                            }
                        }
    } else {
        // coordinate descent: sweep one field with the others held, twice round
        for (int round = 0; round < 2; ++round)
            for (int field = 0; field < 5; ++field) {
                const std::vector<int>& cand = field < 2 ? kz : (field == 2 ? sc_c : (field == 3 ? mc_c : fc));
                for (int v : cand) {
                    evp_tile_config c = cur;
                    int* f = field == 0 ? &c.stress_kz
                                        : field == 1 ? &c.momentum_kz
                                                     : field == 2 ? &c.stress_ctas_per_sm
                                                                  : field == 3 ? &c.momentum_ctas_per_sm : &c.fft_cols;
                    *f = v;
                    double ms = 0.0;
                    if (int r = trial(c, &ms)) return r;
                    if (ms < cur_ms) {
                        cur = c;
                        cur_ms = ms;
                    }
                }
            }
    }
    {
        std::lock_guard<std::mutex> lock(g_cfg_mutex);
        g_cfg[cfg_key(*grid, prec, model)] = cur;
    }
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    if (trials) *trials = n_trials;
    return EVP_OK;
}

}  // extern "C"
