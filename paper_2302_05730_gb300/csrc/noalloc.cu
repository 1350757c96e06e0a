// mcubes_iteration_dev_static: one device-side m-Cubes iteration whose scratch memory lives in
// a fixed array inside this library, so the call itself allocates nothing.
//
// Some callers cannot allocate device memory at the moment they run an iteration:
//  - a host application whose memory pool already owns the whole device;
//  - a latency-critical loop where cudaMalloc or cudaFree would stall or synchronize the device.
// mcubes_iteration_dev needs such a caller to find scratch (the bin-contribution accumulator
// and the two sums). This variant takes it from a file-scope __device__ array instead. Every
// GPU that loads the library holds that array until the process exits.
#include <mutex>

#include "../../include/mcubes.h"
#include "common.cuh"

namespace {

constexpr int kMaxDevices = 64;

// Scratch of one iteration at the largest dimension: C (16 x 500 doubles), then the two sums
// on their own 256-byte line. Keep in step with mcubes_workspace_bytes.
constexpr size_t kStaticScratchBytes = 16 * mcubes::kNB * sizeof(double) + 256;
static_assert(kStaticScratchBytes % 256 == 0, "scratch must be a whole number of 256-byte lines");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, looked up once with that device current.
// In host code the array's name is only a host-side stand-in, never a device address.
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCUBES_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return MCUBES_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MCUBES_OK;
}

}  // namespace

extern "C" size_t mcubes_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int mcubes_iteration_dev_static(int integrand_id, const double *params, int d, int64_t ncall,
                                           uint64_t seed, int iteration, uint32_t job, int adjust,
                                           int precision, const double *d_grid_in, double *d_grid_out,
                                           double *d_result, const double *d_prev,
                                           const mcubes_tuning *tune, void *stream)
{
    if (d < 1 || d > MCUBES_DMAX) return MCUBES_ERR_UNSUPPORTED_DIM;
    const size_t need = mcubes_workspace_bytes(d);
    if (need == 0 || need > kStaticScratchBytes) return MCUBES_ERR_WORKSPACE;
    void *scratch = nullptr;
    const int st = scratch_address(&scratch);
    if (st != MCUBES_OK) return st;
    // A NULL stream means the legacy default stream here. The library's own per-thread stream
    // would be created, and that allocates.
    void *s = stream ? stream : (void *)cudaStreamLegacy;
    return mcubes_iteration_dev(integrand_id, params, d, ncall, seed, iteration, job, adjust, precision,
                                d_grid_in, d_grid_out, d_result, d_prev, scratch, need, tune, s);
}
