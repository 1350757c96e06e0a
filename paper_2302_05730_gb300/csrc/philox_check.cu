// Philox4x32-10 over a list of counters on the device: the library's own generator, its hoisted
// forms (the single-job V-Sample kernels' and the batched kernel's) and, for comparison, the CUDA
// toolkit's cuRAND device function.
#include <curand_kernel.h>

#include "../../include/mcubes.h"
#include "common.cuh"

namespace {

__global__ void philox_own_kernel(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint32_t *out)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        const mcubes::Words4 r = mcubes::philox4x32_10(ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3], k0, k1);
        out[4 * j] = r.x;
        out[4 * j + 1] = r.y;
        out[4 * j + 2] = r.z;
        out[4 * j + 3] = r.w;
    }
}

__global__ void philox_curand_kernel(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint32_t *out)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        uint4 c = make_uint4(ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]);
        uint2 k = make_uint2(k0, k1);
        const uint4 r = curand_Philox4x32_10(c, k);
        out[4 * j] = r.x;
        out[4 * j + 1] = r.y;
        out[4 * j + 2] = r.z;
        out[4 * j + 3] = r.w;
    }
}

// The sampler's hoisted form (philox_prepare, philox_cube, philox_draw): counter word 2 split as
// ctr2_hi = c2 with its low 3 bits cleared and j = those bits.
__global__ void philox_hoisted_kernel(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint32_t *out)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c2 = ctr[4 * j + 2];
        mcubes::PhiloxPre pp;
        mcubes::philox_prepare(pp, k0, k1, c2 & ~7u, ctr[4 * j + 3]);
        const mcubes::PhiloxCube cb = mcubes::philox_cube(ctr[4 * j], pp);
        const mcubes::Words4 r = mcubes::philox_draw(ctr[4 * j + 1], (int)(c2 & 7u), cb, pp);
        out[4 * j] = r.x;
        out[4 * j + 1] = r.y;
        out[4 * j + 2] = r.z;
        out[4 * j + 3] = r.w;
    }
}

// The register form the batched sampler draws with (philox_draw_consts, philox_cube_k, philox_draw_k),
// with the same split of counter word 2.
__global__ void philox_hoisted_reg_kernel(const uint32_t *ctr, uint64_t n, uint32_t k0, uint32_t k1, uint32_t *out)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c2 = ctr[4 * j + 2];
        uint32_t a_j, bk_j;
        mcubes::philox_draw_consts(k0, c2 & ~7u, (int)(c2 & 7u), a_j, bk_j);
        const mcubes::PhiloxCube cb = mcubes::philox_cube_k(ctr[4 * j], ctr[4 * j + 3] ^ k1);
        const mcubes::Words4 r = mcubes::philox_draw_k(ctr[4 * j + 1], a_j, bk_j, cb, k0, k1);
        out[4 * j] = r.x;
        out[4 * j + 1] = r.y;
        out[4 * j + 2] = r.z;
        out[4 * j + 3] = r.w;
    }
}

}  // namespace

extern "C" int mcubes_philox_dev(const uint32_t *d_ctr, uint64_t n, uint64_t seed, int impl, uint32_t *d_out,
                                 void *stream)
{
    if (!d_ctr || !d_out || impl < 0 || impl > 3) return MCUBES_ERR_INVALID_ARG;
    if (n == 0) return MCUBES_OK;
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    cudaStream_t s = (cudaStream_t)stream;
    if (impl == 0) philox_own_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_ctr, n, k0, k1, d_out);
    else if (impl == 1) philox_curand_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_ctr, n, k0, k1, d_out);
    else if (impl == 2) philox_hoisted_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_ctr, n, k0, k1, d_out);
    else philox_hoisted_reg_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_ctr, n, k0, k1, d_out);
    return cudaGetLastError() == cudaSuccess ? MCUBES_OK : MCUBES_ERR_CUDA;
}
