// evp_poisson_solve_static: the fast Poisson solve of evp_poisson_solve without
// any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code running while a CUDA stream is being captured into a graph,
// plugins whose host framework owns every allocation, or processes that run
// under a fixed device-memory budget and must not grow it.  For them this entry
// point keeps all of its scratch (spectral buffer, FFT twiddles, modal
// eigenvalues, Thomas pivots and the sweep buffer) in one file-scope device
// array of fixed size.  The caller passes only the right-hand side and the
// output.
//
// The array (EVP_STATIC_SCRATCH_BYTES) is part of the library image: every GPU
// that loads libevp holds it until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "evp_internal.cuh"

using namespace evp;

namespace evp {
void set_last_error(const std::string& msg);
}

namespace {

constexpr size_t EVP_STATIC_SCRATCH_BYTES = size_t(8) << 20;   // 8 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[EVP_STATIC_SCRATCH_BYTES];

// Per device: the array's device address (looked up with that device current)
// and the configuration whose tables the array currently holds.
struct DeviceSlot {
    bool ready = false;
    unsigned char* base = nullptr;
    bool tables_valid = false;
    evp_grid tables_grid{};
    int tables_precision = -1;
};
DeviceSlot g_slots[MAX_DEVICES];
std::mutex g_slots_mutex;


size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

struct StaticLayout {
    size_t spec, twx, twy, twz, lamx, lamy, lamz, thm, thd, total;
};

StaticLayout layout_of(const evp_grid& g, size_t elt) {
    const int nxh = g.nx / 2 + 1;
    StaticLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.spec = take((size_t)nxh * g.ny * g.nz * 2 * elt);
    L.twx = take((size_t)g.nx * 2 * elt);
    L.twy = take((size_t)g.ny * 2 * elt);
    L.twz = take((size_t)g.nz * 2 * elt);
    L.lamx = take((size_t)nxh * elt);
    L.lamy = take((size_t)g.ny * elt);
    L.lamz = take((size_t)g.nz * elt);
    L.thm = g.walls_y ? take((size_t)(g.nz / 2 + 1) * g.ny * nxh * sizeof(double2)) : 0;
    L.thd = g.walls_y ? take((size_t)2 * nxh * g.ny * g.nz * sizeof(double)) : 0;
    L.total = o;
    return L;
}

// Host-built tables (same definitions as the state-owning path): twiddles
// exp(-2 pi i m/n), eigenvalues (2 - 2 cos(2 pi m/n))/h^2 and, with walls, the
// Thomas pivots (m_j, c'_j) with Neumann rows and the (0, 0) system pinned (FP64
// pairs, or their double-single form for single precision).
template <typename T>
int upload_static_tables(const evp_grid& g, unsigned char* base, const StaticLayout& L, cudaStream_t st) {
    const double dx = g.lx / g.nx, dy = g.ly / g.ny, dz = g.lz / g.nz;
    const int nxh = g.nx / 2 + 1;
    const double twopi = 6.283185307179586476925286766559;
    std::vector<T> buf;
    auto put = [&](size_t off, const std::vector<double>& v) -> cudaError_t {
        buf.assign(v.begin(), v.end());
        // from pageable memory: returns once the data has been staged
        return cudaMemcpyAsync(base + off, buf.data(), buf.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    };
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
    cudaError_t e;
    if ((e = put(L.twx, tw(g.nx))) != cudaSuccess) return EVP_ERR_CUDA;
    if ((e = put(L.twy, tw(g.ny))) != cudaSuccess) return EVP_ERR_CUDA;
    if ((e = put(L.twz, tw(g.nz))) != cudaSuccess) return EVP_ERR_CUDA;
    const std::vector<double> lx = lam(g.nx, nxh, dx);
    if ((e = put(L.lamx, lx)) != cudaSuccess) return EVP_ERR_CUDA;
    if ((e = put(L.lamy, lam(g.ny, g.ny, dy))) != cudaSuccess) return EVP_ERR_CUDA;
    if ((e = put(L.lamz, lam(g.nz, g.nz, dz))) != cudaSuccess) return EVP_ERR_CUDA;
    if (g.walls_y) {
        const std::vector<double> M = thomas_table(g.ny, g.nz, nxh, dy, lx, lam(g.nz, g.nz / 2 + 1, dz));
        // single precision: the double-single table of k_thomas (same bytes per entry)
        const std::vector<float> F = sizeof(T) == 4 ? thomas_table_ds(M) : std::vector<float>();
        const void* src = sizeof(T) == 4 ? static_cast<const void*>(F.data()) : static_cast<const void*>(M.data());
        if ((e = cudaMemcpyAsync(base + L.thm, src, M.size() * sizeof(double), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return EVP_ERR_CUDA;
        // the host vectors end with this scope: the copy from pageable memory has
        // been staged when cudaMemcpyAsync returns
    }
    return EVP_OK;
}

template <typename T>
int solve_static(const evp_grid& g, unsigned char* base, const StaticLayout& L, const T* rhs, T* psi,
                 cudaStream_t st) {
    using CT = typename Cplx<T>::type;
    Geo<T> geo;
    geo.nx = g.nx;
    geo.ny = g.ny;
    geo.nz = g.nz;
    geo.walls = g.walls_y;
    geo.idx = T(g.nx / g.lx);
    geo.idy = T(g.ny / g.ly);
    geo.idz = T(g.nz / g.lz);
    FFTTables<T> tb;
    tb.twx = reinterpret_cast<const CT*>(base + L.twx);
    tb.twy = reinterpret_cast<const CT*>(base + L.twy);
    tb.twz = reinterpret_cast<const CT*>(base + L.twz);
    tb.nrx = fft_radices(g.nx, tb.radx);
    tb.nry = g.walls_y ? 0 : fft_radices(g.ny, tb.rady);
    tb.nrz = fft_radices(g.nz, tb.radz);
    tb.lamx = reinterpret_cast<const T*>(base + L.lamx);
    tb.lamy = reinterpret_cast<const T*>(base + L.lamy);
    tb.lamz = reinterpret_cast<const T*>(base + L.lamz);
    tb.thomas_m = g.walls_y ? reinterpret_cast<const double2*>(base + L.thm) : nullptr;
    tb.thomas_ds = sizeof(T) == 4 ? 1 : 0;
    const double dy = g.ly / g.ny;
    tb.idy2 = 1.0 / (dy * dy);
    PoissonArgs<T> a;
    a.Us = a.Vs = a.Ws = nullptr;
    a.rhs = rhs;
    a.rscale = T(1);
    a.spec = reinterpret_cast<CT*>(base + L.spec);
    a.psi = psi;
    a.norm = g.walls_y ? 1.0 / (double(g.nx) * g.nz) : 1.0 / (double(g.nx) * g.ny * g.nz);
    a.out_scale = g.walls_y ? T(a.norm) : T(1);
    a.scratch = g.walls_y ? reinterpret_cast<double*>(base + L.thd) : nullptr;
    TimingHook none{nullptr, nullptr, nullptr};
    const cudaError_t e = launch_poisson<T>(geo, tb, a, st, none);
    if (e != cudaSuccess) {
        set_last_error(std::string("poisson kernels: ") + cudaGetErrorString(e));
        return EVP_ERR_CUDA;
    }
    return EVP_OK;
}

int static_fail(int code, const std::string& m) {
    set_last_error(m);
    return code;
}

}  // namespace

extern "C" int evp_poisson_solve_static(const evp_grid* grid, int precision, const void* rhs, void* psi,
                                        void* stream) {
    if (!grid || !rhs || !psi) return static_fail(EVP_ERR_ARG, "null argument");
    const evp_grid g = *grid;
    auto fft_ok = [](int n) { return n >= 8 && n <= 512 && is_2a3b(n); };
    if (!fft_ok(g.nx) || g.nx % 2 != 0 || !fft_ok(g.nz) ||
        (g.walls_y ? (g.ny < 4 || g.ny > 512) : !fft_ok(g.ny)) || !(g.lx > 0) || !(g.ly > 0) || !(g.lz > 0))
        return static_fail(EVP_ERR_ARG, "grid sizes must follow the evp_grid rules of evp.h");
    if (precision != EVP_FP64 && precision != EVP_FP32) return static_fail(EVP_ERR_ARG, "bad precision");
    const size_t elt = precision == EVP_FP32 ? 4 : 8;
    const StaticLayout L = layout_of(g, elt);
    if (L.total > EVP_STATIC_SCRATCH_BYTES)
        return static_fail(EVP_ERR_ARG, "grid too large for the static scratch: needs " + std::to_string(L.total) +
                                            " bytes, the array holds " + std::to_string(EVP_STATIC_SCRATCH_BYTES));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(EVP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return static_fail(EVP_ERR_ARG, "device index out of range");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(g_slots_mutex);
    DeviceSlot& slot = g_slots[dev];
    // The host-side name of the array is not a device address: ask the runtime
    // for the address on the current device.  The first call on a device does
    // this lookup (and may load the module); later calls that are not being
    // captured repeat it, which is a table lookup, so that a module reloaded after
    // cudaDeviceReset, whose array lost its contents and may have moved, gets its
    // tables uploaded again.  A captured call uses the address already known.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (st) {
        e = cudaStreamIsCapturing(st, &cap);
        if (e != cudaSuccess)
            return static_fail(EVP_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    }
    if (cap != cudaStreamCaptureStatusNone && !slot.ready)
        return static_fail(EVP_ERR_STATE, "the first call on a device must come before any stream capture");
    void* p = slot.base;
    if (cap == cudaStreamCaptureStatusNone) {
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess)
            return static_fail(EVP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    if (!slot.ready || slot.base != static_cast<unsigned char*>(p)) {
        slot.base = static_cast<unsigned char*>(p);
        slot.tables_valid = false;
        slot.ready = true;
    }
    // compared member by member: a caller's struct may carry arbitrary padding bytes
    const evp_grid& tg = slot.tables_grid;
    const bool same = slot.tables_valid && slot.tables_precision == precision && tg.nx == g.nx && tg.ny == g.ny &&
                      tg.nz == g.nz && tg.lx == g.lx && tg.ly == g.ly && tg.lz == g.lz && tg.walls_y == g.walls_y;
    if (!same && cap != cudaStreamCaptureStatusNone)
        return static_fail(EVP_ERR_STATE, "a call with a new grid or precision cannot be captured: make one "
                                          "call with this grid and precision before the capture");
    if (!same) {
        slot.tables_valid = false;
        const int r = precision == EVP_FP32 ? upload_static_tables<float>(g, slot.base, L, st)
                                            : upload_static_tables<double>(g, slot.base, L, st);
        if (r != EVP_OK) return static_fail(r, "uploading the solver tables failed");
        slot.tables_grid = g;
        slot.tables_precision = precision;
        slot.tables_valid = true;
    }
    if (precision == EVP_FP32)
        return solve_static<float>(g, slot.base, L, static_cast<const float*>(rhs), static_cast<float*>(psi), st);
    return solve_static<double>(g, slot.base, L, static_cast<const double*>(rhs), static_cast<double*>(psi), st);
}
