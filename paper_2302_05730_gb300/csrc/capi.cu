// C ABI of libmcubes.so (declared in include/mcubes.h): argument checks, stratification,
// per-thread device workspace, the iteration loop of m-Cubes (paper Sec. 3.2) and the
// inverse-variance combination of the iteration estimates.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mcubes.h"
#include "internal.h"

using namespace mcubes;

namespace {
thread_local int g_last_cuda_error = 0;

// Allocation fault hook: allocation number g_fail_at (counted from 1 over the library's life)
// fails; 0 = never. MCUBES_FAULT_ALLOC=n arms it at the first allocation.
std::atomic<int64_t> g_alloc_count{0};
std::atomic<int64_t> g_fail_at{0};
std::atomic<int> g_env_read{0};

bool alloc_should_fail()
{
    if (!g_env_read.exchange(1)) {
        const char *e = std::getenv("MCUBES_FAULT_ALLOC");
        if (e && *e) {
            const long long n = std::atoll(e);
            if (n > 0) g_fail_at.store(g_alloc_count.load() + n);
        }
    }
    const int64_t k = g_alloc_count.fetch_add(1) + 1;
    int64_t at = g_fail_at.load();
    return at > 0 && k == at && g_fail_at.compare_exchange_strong(at, 0);
}
}  // namespace

namespace mcubes {

#if MCUBES_CHECKED
// [0] failed index checks, [1] the first failure (site << 48 | index)
__device__ unsigned long long g_bounds_chk[2];
#endif

// The bounds-check words of a checked build on the current device (null otherwise): every
// launch's VsampleParams carries them. The symbol's device address differs per device, so it is
// looked up once per device, with that device current.
unsigned long long *bounds_words()
{
#if MCUBES_CHECKED
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static unsigned long long *addr[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bounds_chk) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        addr[dev] = (unsigned long long *)p;
    }
    return addr[dev];
#else
    return nullptr;
#endif
}

cudaError_t mc_malloc(void **p, size_t bytes)
{
    if (alloc_should_fail()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t mc_malloc_host(void **p, size_t bytes)
{
    if (alloc_should_fail()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return MCUBES_OK;
    g_last_cuda_error = (int)e;
    (void)cudaGetLastError();   // clear the runtime's last-error slot
    return (e == cudaErrorMemoryAllocation) ? MCUBES_ERR_ALLOC : MCUBES_ERR_CUDA;
}

#define MC_TRY(expr)                                   \
    do {                                               \
        const int _st = cuda_status((cudaError_t)(expr)); \
        if (_st != MCUBES_OK) return _st;              \
    } while (0)

constexpr int kGridStride = kNB + 1;

// ---------------------------------------------------------------------------- stratification
// g: the largest integer with 2 g^d <= n (integer arithmetic only); m = g^d; p = max(2, n / m).
static bool pow_at_most(int64_t g, int d, int64_t limit)
{
    int64_t v = 1;
    for (int i = 0; i < d; ++i) {
        if (v > limit / g) return false;
        v *= g;
    }
    return v <= limit;
}

int stratify(int d, int64_t n, int64_t *g, int64_t *m, int64_t *p)
{
    if (d < 1 || d > MCUBES_DMAX) return MCUBES_ERR_UNSUPPORTED_DIM;
    if (n < 2) return MCUBES_ERR_INVALID_ARG;
    const int64_t half = n / 2;
    int64_t lo = 1, hi = half;
    // start the search near the root to keep it short
    const double guess = std::floor(std::pow((double)half, 1.0 / d));
    if (guess >= 1.0 && guess < 9.0e15) {
        int64_t gg = (int64_t)guess;
        while (gg > 1 && !pow_at_most(gg, d, half)) --gg;
        while (pow_at_most(gg + 1, d, half)) ++gg;
        lo = hi = gg;
    }
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (pow_at_most(mid, d, half)) lo = mid; else hi = mid - 1;
    }
    int64_t mm = 1;
    for (int i = 0; i < d; ++i) mm *= lo;
    if (mm > (int64_t)0xFFFFFFFFll) return MCUBES_ERR_INVALID_ARG;
    int64_t pp = n / mm;
    if (pp < 2) pp = 2;
    *g = lo;
    *m = mm;
    *p = pp;
    return MCUBES_OK;
}

// ---------------------------------------------------------------------------- parameters
constexpr double kLog2e = 1.4426950408889634074;
constexpr double kSqrtLog2e = 1.2011224087864498;
constexpr double kTwoPi = 6.283185307179586476925286766559;

int prepare(int fid, const double *params, int d, int64_t ncall, uint64_t seed, int iteration,
            uint32_t job, int adjust, int prec, Problem &pb)
{
    if (d < 1 || d > MCUBES_DMAX) return MCUBES_ERR_UNSUPPORTED_DIM;
    if (fid < 0 || fid >= MCUBES_N_INTEGRANDS) return MCUBES_ERR_UNKNOWN_INTEGRAND;
    if (params == nullptr) return MCUBES_ERR_INVALID_ARG;
    if (prec != MCUBES_FP64 && prec != MCUBES_FP32_EVAL) return MCUBES_ERR_INVALID_ARG;
    if (iteration < 0 || iteration > 0xFFFF) return MCUBES_ERR_INVALID_ARG;
    int st = stratify(d, ncall, &pb.g, &pb.m, &pb.p);
    if (st) return st;
    if (pb.p > 0xFFFFFFFFll) return MCUBES_ERR_INVALID_ARG;
    if (prec == MCUBES_FP32_EVAL && pb.g > (1 << 24)) return MCUBES_ERR_INVALID_ARG;
    for (int i = 0; i < param_len(fid, d); ++i)
        if (!std::isfinite(params[i])) return MCUBES_ERR_INVALID_ARG;

    pb.fid = fid;
    pb.d = d;
    pb.prec = prec;
    VsampleParams &P = pb.P;
    std::memset(&P, 0, sizeof(P));
    P.m = (uint32_t)pb.m;
    P.p = (uint32_t)pb.p;
    P.g = (uint32_t)pb.g;
    P.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    P.key1 = (uint32_t)(seed >> 32);
    P.ctr2_hi = (uint32_t)iteration << 16;
    P.job = job;
    P.adjust = adjust ? 1 : 0;
    P.chk = bounds_words();
    P.R = (double)kNB / (double)pb.g;
    P.R32 = (float)P.R;
    P.ycap = std::nextafter((double)kNB, 0.0);
    P.ycap32 = std::nextafterf((float)kNB, 0.0f);
    P.inv_p = 1.0 / (double)pb.p;
    P.inv_pp1 = 1.0 / ((double)pb.p * (double)(pb.p - 1));
    P.probe_mask = 0xFFFFFFFFu;

    IntegrandParams &ip = P.ip;
    ip.d = d;
    const double *a = params, *u = params + d;
    if (fid == MCUBES_ROTATED_GAUSSIAN) {   // params: M (d x d), then the centre c
        u = params + (size_t)d * d;
        for (int i = 0; i < d * d; ++i) {
            ip.m[i] = params[i];
            ip.fm[i] = (float)(params[i] * kLog2e);
        }
        for (int i = 0; i < d; ++i) {
            ip.u[i] = u[i];
            ip.fu[i] = (float)u[i];
        }
    } else {
        for (int i = 0; i < d; ++i) {
            ip.a[i] = a[i];
            ip.u[i] = u[i];
        }
    }
    if (fid == MCUBES_DOUBLE_GAUSSIAN)
        for (int i = 0; i < d; ++i) ip.b[i] = 1.0 - u[i];
    if (prec == MCUBES_FP64) {
        double s = 1.0;
        for (int i = 0; i < d; ++i) s *= (double)kNB;
        P.fscale = s;   // the Jacobian's nd^d, applied per block
        if (fid == MCUBES_PRODUCT_PEAK)
            for (int i = 0; i < d; ++i) ip.b[i] = 1.0 / (a[i] * a[i]);
    } else {
        double F = 1.0;
        switch (fid) {
        case MCUBES_OSCILLATORY:
            for (int i = 0; i < d; ++i) ip.fa[i] = (float)(a[i] / kTwoPi);
            ip.fc = (float)(u[0] - std::floor(u[0]));
            break;
        case MCUBES_PRODUCT_PEAK:
            for (int i = 0; i < d; ++i) {
                ip.fa[i] = (float)a[i];
                ip.fu[i] = (float)u[i];
                F *= a[i] * a[i];
            }
            break;
        case MCUBES_CORNER_PEAK:
            for (int i = 0; i < d; ++i) ip.fa[i] = (float)a[i];
            break;
        case MCUBES_GAUSSIAN:
            for (int i = 0; i < d; ++i) {
                ip.fa[i] = (float)(a[i] * kSqrtLog2e);
                ip.fu[i] = (float)u[i];
            }
            break;
        case MCUBES_C0:
            for (int i = 0; i < d; ++i) {
                ip.fa[i] = (float)(a[i] * kLog2e);
                ip.fu[i] = (float)u[i];
            }
            break;
        case MCUBES_DISCONTINUOUS: {
            double e = 0.0;
            for (int i = 0; i < d; ++i) {
                const double uc = u[i] < 1.0 ? u[i] : 1.0;
                ip.fa[i] = (float)(a[i] * kLog2e);
                ip.fu[i] = (float)u[i];
                ip.fb[i] = (float)uc;
                e += a[i] * uc;
            }
            F = std::exp(e);
            break;
        }
        case MCUBES_ADDITION:
            break;
        case MCUBES_CONSTANT:
            F = a[0];
            break;
        case MCUBES_DOUBLE_GAUSSIAN:
            for (int i = 0; i < d; ++i) {
                ip.fa[i] = (float)(a[i] * kSqrtLog2e);
                ip.fu[i] = (float)u[i];
                ip.fb[i] = (float)(1.0 - u[i]);
            }
            break;
        case MCUBES_ROTATED_GAUSSIAN:
            break;   // fm, fu set above
        }
        if (!std::isfinite(F)) return MCUBES_ERR_INVALID_ARG;
        P.fscale = F;
    }
    return MCUBES_OK;
}

using Launcher = int (*)(int, const VsampleParams &, const LaunchReq &, cudaStream_t);

static Launcher launcher_for(int prec, int fid)
{
    static const Launcher f64[10] = {launch_vsample_f64_0, launch_vsample_f64_1, launch_vsample_f64_2,
                                     launch_vsample_f64_3, launch_vsample_f64_4, launch_vsample_f64_5,
                                     launch_vsample_f64_6, launch_vsample_f64_7, launch_vsample_f64_8,
                                     launch_vsample_f64_9};
    static const Launcher f32[10] = {launch_vsample_f32_0, launch_vsample_f32_1, launch_vsample_f32_2,
                                     launch_vsample_f32_3, launch_vsample_f32_4, launch_vsample_f32_5,
                                     launch_vsample_f32_6, launch_vsample_f32_7, launch_vsample_f32_8,
                                     launch_vsample_f32_9};
    return prec == MCUBES_FP32_EVAL ? f32[fid] : f64[fid];
}

int make_req(const mcubes_tuning *tune, LaunchReq &req)
{
    int dev = 0;
    MC_TRY(cudaGetDevice(&dev));
    int sms = 0;
    MC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    req.num_sms = sms;
    req.threads = kMaxBlockThreads;
    req.user_threads = 0;
    req.blocks_per_sm = 0;
    req.plain64 = 0;
    if (tune) {
        if (tune->fp64_plain != 0 && tune->fp64_plain != 1) return MCUBES_ERR_INVALID_ARG;
        req.plain64 = tune->fp64_plain;
        if (tune->block_threads) {
            if (tune->block_threads < 64 || tune->block_threads > kMaxBlockThreads || tune->block_threads % 32)
                return MCUBES_ERR_INVALID_ARG;
            req.threads = tune->block_threads;
            req.user_threads = 1;
        }
        if (tune->blocks_per_sm < 0 || tune->blocks_per_sm > 64) return MCUBES_ERR_INVALID_ARG;
        req.blocks_per_sm = tune->blocks_per_sm;
    }
    return MCUBES_OK;
}

int launch_vsample(const Problem &pb, const mcubes_tuning *tune, cudaStream_t s)
{
    LaunchReq req;
    int st = make_req(tune, req);
    if (st) return st;
    return cuda_status((cudaError_t)launcher_for(pb.prec, pb.fid)(pb.d, pb.P, req, s));
}

}  // namespace mcubes

namespace {

// ---------------------------------------------------------------------------- small kernels
__global__ void uniform_grid_kernel(double *grid, int d)
{
    const int n = d * kGridStride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int k = e % kGridStride;
        grid[e] = (double)k / (double)kNB;
    }
}

// result = (sums[0] / m, sums[1] / m^2)
__global__ void finalize_kernel(const double *sums, double *result, double inv_m)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        result[0] = sums[0] * inv_m;
        result[1] = sums[1] * inv_m * inv_m;
    }
}

// ---------------------------------------------------------------------------- workspace
struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    double *d_grid[2] = {nullptr, nullptr};   // ping-pong grids, DMAX x 501
    double *d_C = nullptr;                    // DMAX x 500
    double *d_iter = nullptr;                 // 2 x iter_cap sums
    int iter_cap = 0;
    double *h_pin = nullptr;                  // pinned staging
    size_t h_pin_bytes = 0;

    void release()
    {
        if (device >= 0) {
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(device);
            if (stream) cudaStreamDestroy(stream);
            cudaFree(d_grid[0]);
            cudaFree(d_grid[1]);
            cudaFree(d_C);
            cudaFree(d_iter);
            if (h_pin) cudaFreeHost(h_pin);
            cudaSetDevice(cur);
        }
        *this = Workspace();
    }
};

thread_local Workspace g_ws;

int workspace(int iters, size_t host_bytes, Workspace *&out)
{
    int dev = 0;
    MC_TRY(cudaGetDevice(&dev));
    Workspace &w = g_ws;
    if (w.device != dev) {
        // all or nothing: a failure releases what was made, so the next call starts afresh
        w.release();
        w.device = dev;
        const size_t gb = sizeof(double) * MCUBES_DMAX * kGridStride;
        int st = cuda_status(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
        if (!st) st = cuda_status(mc_malloc((void **)&w.d_grid[0], gb));
        if (!st) st = cuda_status(mc_malloc((void **)&w.d_grid[1], gb));
        if (!st) st = cuda_status(mc_malloc((void **)&w.d_C, sizeof(double) * MCUBES_DMAX * kNB));
        if (st) {
            w.release();
            return st;
        }
    }
    if (iters > w.iter_cap) {
        if (w.d_iter) MC_TRY(cudaFree(w.d_iter));
        w.d_iter = nullptr;
        w.iter_cap = 0;
        MC_TRY(mc_malloc((void **)&w.d_iter, sizeof(double) * 2 * (size_t)iters));
        w.iter_cap = iters;
    }
    if (host_bytes > w.h_pin_bytes) {
        if (w.h_pin) MC_TRY(cudaFreeHost(w.h_pin));
        w.h_pin = nullptr;
        w.h_pin_bytes = 0;
        MC_TRY(mc_malloc_host((void **)&w.h_pin, host_bytes));
        w.h_pin_bytes = host_bytes;
    }
    out = &w;
    return MCUBES_OK;
}

int upload_grid(const double *grid_in, int d, double *d_grid, double *h_stage, cudaStream_t s)
{
    if (grid_in) {
        std::memcpy(h_stage, grid_in, sizeof(double) * d * kGridStride);
        MC_TRY(cudaMemcpyAsync(d_grid, h_stage, sizeof(double) * d * kGridStride, cudaMemcpyHostToDevice, s));
    } else {
        uniform_grid_kernel<<<(d * kGridStride + 255) / 256, 256, 0, s>>>(d_grid, d);
        MC_TRY(cudaGetLastError());
    }
    return MCUBES_OK;
}

bool grid_ok(const double *grid, int d)
{
    for (int i = 0; i < d; ++i) {
        const double *b = grid + (size_t)i * kGridStride;
        if (!(b[0] == 0.0 && b[kNB] == 1.0)) return false;
        for (int k = 0; k < kNB; ++k)
            if (!(b[k + 1] > b[k])) return false;
    }
    return true;
}

// Inverse-variance combination of the iteration estimates.
void combine(const std::vector<double> &I, const std::vector<double> &V, mcubes_result *out)
{
    const int n = (int)I.size();
    int nzero = 0;
    double zsum = 0.0;
    for (int i = 0; i < n; ++i)
        if (V[i] == 0.0) {
            ++nzero;
            zsum += I[i];
        }
    if (nzero > 0) {
        out->estimate = zsum / nzero;
        out->error = 0.0;
        out->chi2_dof = 0.0;
        return;
    }
    double sw = 0.0, swI = 0.0;
    for (int i = 0; i < n; ++i) {
        sw += 1.0 / V[i];
        swI += I[i] / V[i];
    }
    const double Ibar = swI / sw;
    double chi = 0.0;
    for (int i = 0; i < n; ++i) chi += (I[i] - Ibar) * (I[i] - Ibar) / V[i];
    out->estimate = Ibar;
    out->error = 1.0 / std::sqrt(sw);
    out->chi2_dof = n > 1 ? chi / (double)(n - 1) : 0.0;
}

}  // namespace

// ============================================================================ exported calls
extern "C" {

const char *mcubes_status_string(int status)
{
    switch (status) {
    case MCUBES_OK: return "ok";
    case MCUBES_ERR_INVALID_ARG: return "invalid argument";
    case MCUBES_ERR_UNSUPPORTED_DIM: return "unsupported dimension (1..16)";
    case MCUBES_ERR_UNKNOWN_INTEGRAND: return "unknown integrand id";
    case MCUBES_ERR_CUDA: return "CUDA runtime error";
    case MCUBES_ERR_ALLOC: return "allocation failed";
    case MCUBES_ERR_NONFINITE: return "integrand produced a non-finite value";
    case MCUBES_ERR_TIMEOUT: return "device-side wait timed out";
    case MCUBES_ERR_WORKSPACE: return "workspace too small or misaligned";
    default: return "unknown status";
    }
}

int mcubes_last_cuda_error(void) { return g_last_cuda_error; }

void mcubes_shutdown(void) { g_ws.release(); }

int64_t mcubes_checked_violations(int reset, int64_t *first)
{
#if MCUBES_CHECKED
    unsigned long long *w = bounds_words();
    if (!w) return -1;
    unsigned long long h[2] = {0ull, 0ull};
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h, w, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    if (first) *first = (int64_t)h[1];
    if (reset) {
        const unsigned long long z[2] = {0ull, 0ull};
        if (cudaMemcpy(w, z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) (void)cudaGetLastError();
    }
    return (int64_t)h[0];
#else
    (void)reset;
    if (first) *first = 0;
    return -1;
#endif
}

int64_t mcubes_fail_alloc(int64_t n)
{
    g_env_read.store(1);   // an explicit call overrides the environment
    const int64_t made = g_alloc_count.load();
    g_fail_at.store(n > 0 ? made + n : 0);
    return made;
}

int mcubes_stratify(int d, int64_t ncall, int64_t *g, int64_t *m, int64_t *p)
{
    if (!g || !m || !p) return MCUBES_ERR_INVALID_ARG;
    return stratify(d, ncall, g, m, p);
}

}  // extern "C"

namespace {

// Iterations [it_begin, it_end) of an integration of itmax iterations whose first iter_adjust
// iterations refine the grid. grid_in: the grid before it_begin (NULL: uniform). prev_I: the
// estimate of iteration it_begin - 1 (0: none); it only sets the FP32-eval histogram scale.
// Writes the per-iteration (I, Var) into I, V and, if grid_out, the grid after the range.
int run_range(Problem &pb, int itmax, int iter_adjust, int it_begin, int it_end, const double *grid_in,
              double prev_I, const mcubes_tuning *tune, void *stream, std::vector<double> &I,
              std::vector<double> &V, double *grid_out)
{
    const int d = pb.d;
    const int n = it_end - it_begin;
    Workspace *w = nullptr;
    const size_t host_bytes = sizeof(double) * (2 * (size_t)(n + 1) + (size_t)d * kGridStride);
    int st = workspace(n + 1, host_bytes, w);
    if (st) return st;
    cudaStream_t s = stream ? (cudaStream_t)stream : w->stream;
    const double m = (double)pb.m;

    int cur = 0;
    if ((st = upload_grid(grid_in, d, w->d_grid[0], w->h_pin, s))) return st;
    // slot 0 holds the previous iteration's raw sums (for the FP32 histogram scale)
    if ((st = cuda_status(cudaStreamSynchronize(s)))) return st;   // the staging buffer is reused below
    w->h_pin[0] = prev_I * m;
    w->h_pin[1] = 0.0;
    if ((st = cuda_status(cudaMemsetAsync(w->d_iter, 0, sizeof(double) * 2 * (n + 1), s)))) return st;
    if ((st = cuda_status(cudaMemcpyAsync(w->d_iter, w->h_pin, sizeof(double) * 2, cudaMemcpyHostToDevice, s))))
        return st;
    for (int it = it_begin; it < it_end; ++it) {
        const int slot = it - it_begin + 1;
        const int adjust = it < iter_adjust;
        VsampleParams &P = pb.P;
        P.grid = w->d_grid[cur];
        P.C = w->d_C;
        P.sums = w->d_iter + 2 * slot;
        P.prev = (it > it_begin || prev_I != 0.0) ? w->d_iter + 2 * (slot - 1) : nullptr;   // raw sums
        P.prev_scale = 1.0 / m;
        P.adjust = adjust;
        P.ctr2_hi = (uint32_t)it << 16;
        if (adjust) {
            if ((st = cuda_status(cudaMemsetAsync(w->d_C, 0, sizeof(double) * d * kNB, s)))) return st;
        }
        if ((st = launch_vsample(pb, tune, s))) return st;
        if (adjust && it + 1 < itmax) {
            if ((st = cuda_status((cudaError_t)launch_rebin(d, w->d_grid[cur], w->d_C, w->d_grid[1 - cur], 1.5, s))))
                return st;
            cur = 1 - cur;
        }
    }
    double *h_iter = w->h_pin;
    double *h_grid = w->h_pin + 2 * (n + 1);
    if ((st = cuda_status(cudaMemcpyAsync(h_iter, w->d_iter, sizeof(double) * 2 * (n + 1), cudaMemcpyDeviceToHost, s))))
        return st;
    if (grid_out) {
        if ((st = cuda_status(cudaMemcpyAsync(h_grid, w->d_grid[cur], sizeof(double) * d * kGridStride,
                                              cudaMemcpyDeviceToHost, s))))
            return st;
    }
    if ((st = cuda_status(cudaStreamSynchronize(s)))) return st;
    I.assign(n, 0.0);
    V.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        I[k] = h_iter[2 * (k + 1)] / m;
        V[k] = h_iter[2 * (k + 1) + 1] / (m * m);
        if (!std::isfinite(I[k]) || !std::isfinite(V[k])) return MCUBES_ERR_NONFINITE;
    }
    if (grid_out) std::memcpy(grid_out, h_grid, sizeof(double) * d * kGridStride);
    return MCUBES_OK;
}

}  // namespace

extern "C" {

namespace {

// Run log: with MCUBES_LOG=<file> in the environment, every whole-run call appends one JSON line
// per iteration (its estimate and sigma, and the running inverse-variance combination with its
// chi^2/dof) and a summary line (the result, wall time, samples/s).
void json_num(std::string &o, double v)
{
    char b[40];
    if (std::isfinite(v)) {
        std::snprintf(b, sizeof(b), "%.17g", v);
        o += b;
    } else {
        o += "null";
    }
}

void log_run(const char *call, const Problem &pb, int itmax, int iter_adjust, int it_begin,
             const std::vector<double> &I, const std::vector<double> &V, const mcubes_result *res, double ms)
{
    const char *path = std::getenv("MCUBES_LOG");
    if (!path || !*path) return;
    std::string o;
    char b[256];
    const double samples = (double)pb.m * (double)pb.p;
    double sw = 0.0, swI = 0.0, swI2 = 0.0;
    for (size_t k = 0; k < I.size(); ++k) {
        const int it = it_begin + (int)k;
        std::snprintf(b, sizeof(b), "{\"event\": \"iteration\", \"call\": \"%s\", \"it\": %d, \"adjust\": %s, \"I\": ", call,
                      it, it < iter_adjust ? "true" : "false");
        o += b;
        json_num(o, I[k]);
        o += ", \"sigma\": ";
        json_num(o, std::sqrt(V[k]));
        // running combination over this call's iterations so far
        if (V[k] > 0.0) {
            const double w = 1.0 / V[k];
            sw += w;
            swI += w * I[k];
            swI2 += w * I[k] * I[k];
        }
        const double est = sw > 0.0 ? swI / sw : I[k];
        const double chi2 = k > 0 && sw > 0.0 ? std::max(0.0, swI2 - swI * swI / sw) / (double)k : 0.0;
        o += ", \"running_estimate\": ";
        json_num(o, est);
        o += ", \"running_error\": ";
        json_num(o, sw > 0.0 ? 1.0 / std::sqrt(sw) : 0.0);
        o += ", \"running_chi2_dof\": ";
        json_num(o, chi2);
        std::snprintf(b, sizeof(b), ", \"samples\": %.0f}\n", samples);
        o += b;
    }
    std::snprintf(b, sizeof(b),
                  "{\"event\": \"run\", \"call\": \"%s\", \"integrand\": %d, \"d\": %d, \"samples_per_iter\": %.0f, "
                  "\"itmax\": %d, \"iter_adjust\": %d, \"iterations\": %d, \"precision\": \"%s\", \"ms\": ",
                  call, pb.fid, pb.d, samples, itmax, iter_adjust, (int)I.size(),
                  pb.prec == MCUBES_FP32_EVAL ? "fp32_eval" : "fp64");
    o += b;
    json_num(o, ms);
    o += ", \"samples_per_s\": ";
    json_num(o, ms > 0.0 ? samples * (double)I.size() / (ms * 1e-3) : 0.0);
    if (res) {
        o += ", \"estimate\": ";
        json_num(o, res->estimate);
        o += ", \"error\": ";
        json_num(o, res->error);
        o += ", \"chi2_dof\": ";
        json_num(o, res->chi2_dof);
    }
    o += "}\n";
    if (FILE *f = std::fopen(path, "a")) {
        std::fwrite(o.data(), 1, o.size(), f);
        std::fclose(f);
    }
}

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

int mcubes_integrate_ex(int integrand_id, const double *params, int d, int64_t ncall, int itmax,
                        int iter_adjust, uint64_t seed, int precision, const mcubes_tuning *tune,
                        void *stream, double *iter_out, const double *grid_in, double *grid_out,
                        mcubes_result *out)
{
    if (out) std::memset(out, 0, sizeof(*out));
    int st = MCUBES_OK;
    Problem pb;
    if (!out) st = MCUBES_ERR_INVALID_ARG;
    else if (itmax < 1 || itmax > 0xFFFF || iter_adjust < 0 || iter_adjust > itmax) st = MCUBES_ERR_INVALID_ARG;
    if (!st) st = prepare(integrand_id, params, d, ncall, seed, 0, 0, iter_adjust > 0, precision, pb);
    if (!st && grid_in && !grid_ok(grid_in, d)) st = MCUBES_ERR_INVALID_ARG;
    std::vector<double> I, V;
    const auto t0 = std::chrono::steady_clock::now();
    if (!st) st = run_range(pb, itmax, iter_adjust, 0, itmax, grid_in, 0.0, tune, stream, I, V, grid_out);
    const double ms = ms_since(t0);
    if (st) {
        if (out) out->status = st;
        return st;
    }
    if (iter_out)
        for (int it = 0; it < itmax; ++it) {
            iter_out[2 * it] = I[it];
            iter_out[2 * it + 1] = V[it];
        }
    combine(I, V, out);
    out->iters_done = itmax;
    out->samples_per_iter = pb.m * pb.p;
    out->status = MCUBES_OK;
    log_run("integrate", pb, itmax, iter_adjust, 0, I, V, out, ms);
    return MCUBES_OK;
}

int mcubes_integrate_range(int integrand_id, const double *params, int d, int64_t ncall, int itmax,
                           int iter_adjust, int it_begin, int it_end, uint64_t seed, int precision,
                           const double *grid_in, double prev_estimate, double *grid_out, double *iter_out,
                           void *stream)
{
    if (itmax < 1 || itmax > 0xFFFF || iter_adjust < 0 || iter_adjust > itmax) return MCUBES_ERR_INVALID_ARG;
    if (it_begin < 0 || it_end <= it_begin || it_end > itmax || !iter_out) return MCUBES_ERR_INVALID_ARG;
    if (!std::isfinite(prev_estimate)) return MCUBES_ERR_INVALID_ARG;
    if (grid_in == nullptr && it_begin > 0) return MCUBES_ERR_INVALID_ARG;   // a resumed range needs its grid
    Problem pb;
    int st = prepare(integrand_id, params, d, ncall, seed, 0, 0, iter_adjust > 0, precision, pb);
    if (st) return st;
    if (grid_in && !grid_ok(grid_in, d)) return MCUBES_ERR_INVALID_ARG;
    std::vector<double> I, V;
    const auto t0 = std::chrono::steady_clock::now();
    st = run_range(pb, itmax, iter_adjust, it_begin, it_end, grid_in, prev_estimate, nullptr, stream, I, V, grid_out);
    const double ms = ms_since(t0);
    if (st) return st;
    for (int k = 0; k < it_end - it_begin; ++k) {
        iter_out[2 * k] = I[k];
        iter_out[2 * k + 1] = V[k];
    }
    log_run("integrate_range", pb, itmax, iter_adjust, it_begin, I, V, nullptr, ms);
    return MCUBES_OK;
}

int mcubes_combine(const double *iter, int n, int skip, mcubes_result *out)
{
    if (!iter || !out || n < 1 || skip < 0 || skip >= n) return MCUBES_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    std::vector<double> I, V;
    for (int k = skip; k < n; ++k) {
        if (!std::isfinite(iter[2 * k]) || !std::isfinite(iter[2 * k + 1]) || iter[2 * k + 1] < 0.0) {
            out->status = MCUBES_ERR_INVALID_ARG;
            return MCUBES_ERR_INVALID_ARG;
        }
        I.push_back(iter[2 * k]);
        V.push_back(iter[2 * k + 1]);
    }
    combine(I, V, out);
    out->iters_done = n - skip;
    out->status = MCUBES_OK;
    return MCUBES_OK;
}

int mcubes_integrate(int integrand_id, const double *params, int d, int64_t ncall, int itmax,
                     int iter_adjust, uint64_t seed, mcubes_result *out)
{
    return mcubes_integrate_ex(integrand_id, params, d, ncall, itmax, iter_adjust, seed, MCUBES_FP64,
                               nullptr, nullptr, nullptr, nullptr, nullptr, out);
}

int mcubes_vsample_once(int integrand_id, const double *params, int d, int64_t ncall, uint64_t seed,
                        int iteration, uint32_t job, int adjust, int precision, const double *grid_in,
                        double *grid_out, double *C_out, double *I_out, double *var_out)
{
    Problem pb;
    int st = prepare(integrand_id, params, d, ncall, seed, iteration, job, adjust, precision, pb);
    if (st) return st;
    if (!I_out || !var_out) return MCUBES_ERR_INVALID_ARG;
    if (grid_in && !grid_ok(grid_in, d)) return MCUBES_ERR_INVALID_ARG;
    Workspace *w = nullptr;
    const size_t nb = (size_t)d * kGridStride, nc = (size_t)d * kNB;
    if ((st = workspace(1, sizeof(double) * (nb + nc + 2 + nb), w))) return st;
    cudaStream_t s = w->stream;
    if ((st = upload_grid(grid_in, d, w->d_grid[0], w->h_pin, s))) return st;
    MC_TRY(cudaMemsetAsync(w->d_iter, 0, sizeof(double) * 2, s));
    if (adjust) MC_TRY(cudaMemsetAsync(w->d_C, 0, sizeof(double) * nc, s));
    VsampleParams &P = pb.P;
    P.grid = w->d_grid[0];
    P.C = w->d_C;
    P.sums = w->d_iter;
    if ((st = launch_vsample(pb, nullptr, s))) return st;
    if (adjust && grid_out) {
        MC_TRY(launch_rebin(d, w->d_grid[0], w->d_C, w->d_grid[1], 1.5, s));
    }
    double *h_sums = w->h_pin + nb;
    double *h_C = h_sums + 2;
    double *h_grid = h_C + nc;
    MC_TRY(cudaMemcpyAsync(h_sums, w->d_iter, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    if (adjust && C_out) MC_TRY(cudaMemcpyAsync(h_C, w->d_C, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    if (adjust && grid_out)
        MC_TRY(cudaMemcpyAsync(h_grid, w->d_grid[1], sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    MC_TRY(cudaStreamSynchronize(s));
    const double m = (double)pb.m;
    const double I = h_sums[0] / m, V = h_sums[1] / (m * m);
    if (!std::isfinite(I) || !std::isfinite(V)) return MCUBES_ERR_NONFINITE;
    *I_out = I;
    *var_out = V;
    if (adjust && C_out) std::memcpy(C_out, h_C, sizeof(double) * nc);
    if (adjust && grid_out) std::memcpy(grid_out, h_grid, sizeof(double) * nb);
    return MCUBES_OK;
}

int mcubes_vsample_dev(int integrand_id, const double *params, int d, int64_t ncall, uint64_t seed,
                       int iteration, uint32_t job, int adjust, int precision, const double *d_grid,
                       double *d_C, double *d_sums, const double *d_prev, double *d_probe,
                       int probe_shift, const mcubes_tuning *tune, void *stream)
{
    Problem pb;
    int st = prepare(integrand_id, params, d, ncall, seed, iteration, job, adjust, precision, pb);
    if (st) return st;
    if (!d_grid || !d_sums || (adjust && !d_C)) return MCUBES_ERR_INVALID_ARG;
    if (probe_shift < 0 || probe_shift > 31) return MCUBES_ERR_INVALID_ARG;
    VsampleParams &P = pb.P;
    P.grid = d_grid;
    P.C = d_C;
    P.sums = d_sums;
    P.prev = d_prev;
    P.prev_scale = 1.0;
    P.probe = d_probe;
    P.probe_shift = (uint32_t)probe_shift;
    P.probe_mask = d_probe ? ((probe_shift == 0) ? 0u : ((1u << probe_shift) - 1u)) : 0xFFFFFFFFu;
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {
        Workspace *w = nullptr;
        if ((st = workspace(1, 0, w))) return st;
        s = w->stream;
    }
    return launch_vsample(pb, tune, s);
}

int mcubes_rebin_dev(int d, const double *d_grid_in, const double *d_C, double *d_grid_out, void *stream)
{
    if (d < 1 || d > MCUBES_DMAX) return MCUBES_ERR_UNSUPPORTED_DIM;
    if (!d_grid_in || !d_C || !d_grid_out || d_grid_in == d_grid_out) return MCUBES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {
        Workspace *w = nullptr;
        int st = workspace(1, 0, w);
        if (st) return st;
        s = w->stream;
    }
    return cuda_status((cudaError_t)launch_rebin(d, d_grid_in, d_C, d_grid_out, 1.5, s));
}

size_t mcubes_workspace_bytes(int d)
{
    if (d < 1 || d > MCUBES_DMAX) return 0;
    const size_t c = sizeof(double) * (size_t)d * kNB;
    const size_t c_al = (c + 255) & ~(size_t)255;
    return c_al + 256;   // C, then the two sums
}

int mcubes_iteration_dev(int integrand_id, const double *params, int d, int64_t ncall, uint64_t seed,
                         int iteration, uint32_t job, int adjust, int precision, const double *d_grid_in,
                         double *d_grid_out, double *d_result, const double *d_prev, void *d_workspace,
                         size_t workspace_bytes, const mcubes_tuning *tune, void *stream)
{
    Problem pb;
    int st = prepare(integrand_id, params, d, ncall, seed, iteration, job, adjust, precision, pb);
    if (st) return st;
    if (!d_grid_in || !d_grid_out || !d_result || d_grid_in == d_grid_out) return MCUBES_ERR_INVALID_ARG;
    const size_t need = mcubes_workspace_bytes(d);
    if (!d_workspace || workspace_bytes < need || ((uintptr_t)d_workspace & 255u)) return MCUBES_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {
        Workspace *w = nullptr;
        if ((st = workspace(1, 0, w))) return st;
        s = w->stream;
    }
    double *C = (double *)d_workspace;
    double *sums = (double *)((char *)d_workspace + (need - 256));
    MC_TRY(cudaMemsetAsync(d_workspace, 0, need, s));
    VsampleParams &P = pb.P;
    P.grid = d_grid_in;
    P.C = C;
    P.sums = sums;
    P.prev = d_prev;
    P.prev_scale = 1.0;
    if ((st = launch_vsample(pb, tune, s))) return st;
    if (adjust) {
        MC_TRY(launch_rebin(d, d_grid_in, C, d_grid_out, 1.5, s));
    } else {
        MC_TRY(cudaMemcpyAsync(d_grid_out, d_grid_in, sizeof(double) * d * kGridStride, cudaMemcpyDeviceToDevice, s));
    }
    finalize_kernel<<<1, 32, 0, s>>>(sums, d_result, 1.0 / (double)pb.m);
    MC_TRY(cudaGetLastError());
    return MCUBES_OK;
}

}  // extern "C"
