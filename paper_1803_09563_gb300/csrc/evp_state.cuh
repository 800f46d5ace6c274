// Host-side layout of a simulation state (the evp_state of evp.h) and the small
// helpers that turn it into kernel arguments, shared by the state's own entry
// points (evp_abi.cu) and the batched step (evp_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "evp_internal.cuh"

struct evp_state_s {
    evp_grid g;
    evp_model model;
    evp_params prm;
    bool fp32;
    size_t elt;          // bytes per element
    size_t N;            // cells
    int nxh;
    cudaStream_t st;
    bool own_stream;
    char* arena;
    size_t arena_bytes;
    bool own_arena;
    // field storage (element type = precision)
    void* U[2];
    void* V[2];
    void* W[2];
    void* B[2][6];
    void* RT[6];
    void* NH[3];
    void* S[6];          // RK3 with a stress (not soft particles): tau^k + tau^{k-1}, stress -> momentum
    void* P;
    void* PSI;
    void* spec;
    // tables
    void* twx;
    void* twy;
    void* twz;
    void* lamx;
    void* lamy;
    void* lamz;
    void* trig;
    double2* thomas_m;
    double* thomas_d;
    unsigned* d_status;
    unsigned long long* d_maxdiv;
    void* diag;          // evp_diagnostics: DIAG_BLOCKS block partials, then the folded record
    // two-phase (AB2) fields
    bool ab2;
    void* PHI;
    void* PHI0;
    void* PHIA;
    void* PHIB;
    void* HF;
    void* NRM[3];
    void* FC[3];
    void* SOL[3];        // penalization: solid fractions at the velocity nodes
    void* POLD;          // AB2 with a density contrast: p^{n-1}
    double* partials;
    double* mean_1mH;
    double* mass;        // mass correction: 2 x block partials, v0, d
    void* PHS[2];        // soft particles: solid fraction, buffer cb = current level
    void* PHSH;          // soft particles: history of its right-hand side
    double2* helm[3][2]; // implicit viscous, walls: Thomas tables per substep, (u/w, v)
    double helm_dt;      // dt the Helmholtz tables were built for
    // rigid particles (discrete-forcing IBM): one device block holding the arrays below
    int n_part, n_lag, ibm_iters;
    void* ibm_block;
    double *i_off, *i_dvl, *i_centre, *i_vel, *i_omg, *i_Facc, *i_dF, *i_force, *i_rad, *i_dens, *i_int;
    int *i_owner, *i_start;
    int any_free;
    long long nstep;     // AB2 steps taken
    int cu, cb;          // current velocity / B buffer
    // CUDA-graph replay of evp_step: one executable graph per parity of the B
    // buffer at the start of the step (the three substeps flip it each time)
    bool use_graph;
    bool pdl;            // programmatic dependent launch of the step's kernels
    bool nvtx;           // NVTX ranges around steps, substeps and kernel launches
    struct StepGraph {
        bool valid;
        double dt;
        int cb_after;
        cudaGraphExec_t exec;
    } graphs[2];
    evp::ModelConst mc;
    // batch membership (evp_batch_admit): the batch and the stream its steps run on
    void* batch;
    cudaStream_t batch_st;
    // timing
    bool timing;
    std::vector<cudaEvent_t> ev_free;
    struct Pend {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<Pend> pending;
    cudaEvent_t cur_start;
    double ms[evp::K_COUNT];
    long long launches[evp::K_COUNT];
};

namespace evp {

// Wray's low-storage RK3 constants (Eq. RK)
constexpr double RK_ALPHA[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
constexpr double RK_ZETA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
constexpr double RK_XI[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

template <typename T>
inline Geo<T> geo_of(const evp_state* s) {
    Geo<T> g;
    g.nx = s->g.nx;
    g.ny = s->g.ny;
    g.nz = s->g.nz;
    g.walls = s->g.walls_y;
    g.idx = T(s->g.nx / s->g.lx);
    g.idy = T(s->g.ny / s->g.ly);
    g.idz = T(s->g.nz / s->g.lz);
    return g;
}

template <typename T>
inline FFTTables<T> tables_of(const evp_state* s) {
    using CT = typename Cplx<T>::type;
    FFTTables<T> t;
    t.twx = static_cast<const CT*>(s->twx);
    t.twy = static_cast<const CT*>(s->twy);
    t.twz = static_cast<const CT*>(s->twz);
    t.nrx = fft_radices(s->g.nx, t.radx);
    t.nry = s->g.walls_y ? 0 : fft_radices(s->g.ny, t.rady);
    t.nrz = fft_radices(s->g.nz, t.radz);
    t.lamx = static_cast<const T*>(s->lamx);
    t.lamy = static_cast<const T*>(s->lamy);
    t.lamz = static_cast<const T*>(s->lamz);
    t.thomas_m = s->thomas_m;
    t.thomas_ds = s->fp32 && !s->prm.thomas_fp64;
    const double dy = s->g.ly / s->g.ny;
    t.idy2 = 1.0 / (dy * dy);
    return t;
}

template <typename T>
inline double poisson_norm(const evp_state* s) {
    const evp_grid& g = s->g;
    return g.walls_y ? 1.0 / (double(g.nx) * g.nz) : 1.0 / (double(g.nx) * g.ny * g.nz);
}

void set_last_error(const std::string& msg);

}  // namespace evp
