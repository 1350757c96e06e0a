// Unit-rate microbenchmarks (mcubes_unit_rates): the per-SM throughput of the operations the
// V-Sample kernels are built from, measured on the current device, in operations (lanes) per SM
// per clock. They back the kernels' bounds: the random shared-memory accesses of the histogram
// and the grid table, Philox4x32-10, the FP32 and FP64 pipes and the SFU.
//
// Each probe runs 8 independent dependency chains per thread over a resident grid (the SM count
// times 4 blocks of 256 threads), so issue and pipe throughput, not latency, set its time. Every
// shared index is masked into its array.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mcubes.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kIters = 512;
constexpr int kThreads = 256;
constexpr int kBins = 500;    // bins per axis, as the histogram
constexpr int kAxes = 8;
constexpr int kUnitRates = 12;

__device__ __forceinline__ uint32_t lcg(uint32_t s) { return s * 1664525u + 1013904223u; }
// a bin index in [0, kBins) from the top 16 bits of a 32-bit state
__device__ __forceinline__ int bin_of(uint32_t s) { return (int)((((s >> 16) & 0xFFFFu) * (uint32_t)kBins) >> 16); }

__global__ void k_ffma(float *out, float a, float b)
{
    float x[8];
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(float *out, double a, double b)
{
    double x[8];
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void k_ex2(float *out)
{
    float x[8];
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-6f - 0.5f * i;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = -exp2f(x[i]);
    }
    float s = 0.f;
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Philox4x32-10 calls: two independent calls an iteration (a d = 8 sample's draws)
__global__ void k_philox(float *out, uint32_t k0, uint32_t k1)
{
    uint32_t acc = 0;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t it = 0; it < kIters / 4; ++it) {
        const mcubes::Words4 a = mcubes::philox4x32_10(t, it, 0u, 7u, k0, k1);
        const mcubes::Words4 b = mcubes::philox4x32_10(t, it, 1u, 7u, k0, k1);
        acc ^= a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
    }
    out[t] = (float)acc;
}

// random 8-byte gathers from a d x 500 float2 table: one an axis, chained through an FMA
__global__ void k_gather(float *out, uint32_t seed)
{
    extern __shared__ __align__(16) unsigned char sm[];
    float2 *tab = reinterpret_cast<float2 *>(sm);
    for (int e = threadIdx.x; e < kAxes * kBins; e += blockDim.x) tab[e] = make_float2(e * 1e-4f, 1.0f + e * 1e-7f);
    __syncthreads();
    uint32_t s = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu);
    float acc = 0.f;
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int i = 0; i < kAxes; ++i) {
            s = lcg(s);
            const float2 v = tab[i * kBins + bin_of(s)];
            acc = fmaf(acc, v.y, v.x);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// the same gathers through the L1 data cache (read-only global loads of an 8 x 500 table), and a
// mix: axes 0-3 from shared memory, axes 4-7 through L1
template <bool kMix>
__global__ void k_gather_l1(float *out, const float2 *__restrict__ gtab, uint32_t seed)
{
    extern __shared__ __align__(16) unsigned char sm[];
    float2 *tab = reinterpret_cast<float2 *>(sm);
    if (kMix)
        for (int e = threadIdx.x; e < kAxes * kBins; e += blockDim.x) tab[e] = make_float2(e * 1e-4f, 1.0f + e * 1e-7f);
    __syncthreads();
    uint32_t s = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu);
    float acc = 0.f;
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int i = 0; i < kAxes; ++i) {
            s = lcg(s);
            const int e = i * kBins + bin_of(s);
            const float2 v = (kMix && i < kAxes / 2) ? tab[e] : __ldg(&gtab[e]);
            acc = fmaf(acc, v.y, v.x);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void k_fill_table(float2 *gtab)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kAxes * kBins) gtab[e] = make_float2(e * 1e-4f, 1.0f + e * 1e-7f);
}

// random FP32 shared atomics into one d x 500 histogram
__global__ void k_atom_f32(float *out, uint32_t seed)
{
    extern __shared__ __align__(16) unsigned char sm[];
    float *h = reinterpret_cast<float *>(sm);
    for (int e = threadIdx.x; e < kAxes * kBins; e += blockDim.x) h[e] = 0.f;
    __syncthreads();
    uint32_t s = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu);
    for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
        for (int i = 0; i < kAxes; ++i) {
            s = lcg(s);
            atomicAdd(&h[i * kBins + bin_of(s)], 1.0f);
        }
    }
    __syncthreads();
    float acc = 0.f;
    for (int e = threadIdx.x; e < kAxes * kBins; e += blockDim.x) acc += h[e];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// the fixed-point histogram's update: a u32 atomic with its old value into one of 8
// lane-interleaved low-word copies, the carry into one high word per bin
__global__ void k_atom_u32x8(float *out, uint32_t seed)
{
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t *lo = reinterpret_cast<uint32_t *>(sm);
    uint32_t *hi = lo + kAxes * kBins * 8;
    for (int e = threadIdx.x; e < kAxes * kBins * 9; e += blockDim.x) lo[e] = 0u;
    __syncthreads();
    const int g = threadIdx.x & 7;
    uint32_t s = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu);
    for (int it = 0; it < kIters / 8; ++it) {
        const uint32_t v = (s >> 4) | 1u;
#pragma unroll
        for (int i = 0; i < kAxes; ++i) {
            s = lcg(s);
            const int b = i * kBins + bin_of(s);
            const uint32_t old = atomicAdd(&lo[b * 8 + g], v);
            if (old + v < old) atomicAdd(&hi[b], 1u);
        }
    }
    __syncthreads();
    float acc = 0.f;
    for (int e = threadIdx.x; e < kAxes * kBins * 9; e += blockDim.x) acc += (float)lo[e];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// 64-bit fixed-point adds without a returned value (red.shared.add.u64) into R lane-interleaved
// copies of the 8 x 500 histogram (copy g = lane mod R holds bin e at word e R + g)
template <int R>
__global__ void k_red_u64(float *out, uint32_t seed)
{
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *h = reinterpret_cast<unsigned long long *>(sm);
    for (int e = threadIdx.x; e < kAxes * kBins * R; e += blockDim.x) h[e] = 0ull;
    __syncthreads();
    const int g = threadIdx.x & (R - 1);
    uint32_t s = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu);
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(h);
    for (int it = 0; it < kIters / 8; ++it) {
        const unsigned long long v = ((unsigned long long)(s >> 4) << 12) | 1ull;
#pragma unroll
        for (int i = 0; i < kAxes; ++i) {
            s = lcg(s);
            const uint32_t a = base + (uint32_t)(((i * kBins + bin_of(s)) * R + g) * 8);
            asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
        }
    }
    __syncthreads();
    float acc = 0.f;
    for (int e = threadIdx.x; e < kAxes * kBins * R; e += blockDim.x) acc += (float)h[e];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// u32 adds without a returned value (red.shared.add.u32) into 8 lane-interleaved copies: the
// fixed-point update without its carry
__global__ void k_red_u32x8(float *out, uint32_t seed)
{
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t *h = reinterpret_cast<uint32_t *>(sm);
    for (int e = threadIdx.x; e < kAxes * kBins * 8; e += blockDim.x) h[e] = 0u;
    __syncthreads();
    const int g = threadIdx.x & 7;
    uint32_t s = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu);
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(h);
    for (int it = 0; it < kIters / 8; ++it) {
        const uint32_t v = (s >> 4) | 1u;
#pragma unroll
        for (int i = 0; i < kAxes; ++i) {
            s = lcg(s);
            const uint32_t a = base + (uint32_t)(((i * kBins + bin_of(s)) * 8 + g) * 4);
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
        }
    }
    __syncthreads();
    float acc = 0.f;
    for (int e = threadIdx.x; e < kAxes * kBins * 8; e += blockDim.x) acc += (float)h[e];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

struct Probe {
    int threads, blocks_per_sm;
    size_t smem;
    double ops_per_thread;
};

template <typename Launch>
double time_probe(const Probe &p, int sms, double clk_hz, float *buf, Launch launch, int &st)
{
    const unsigned blocks = (unsigned)(sms * p.blocks_per_sm);
    launch(blocks, p.threads, p.smem, buf);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaEventRecord(e0);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        launch(blocks, p.threads, p.smem, buf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        st = mcubes::cuda_status(e);
        return 0.0;
    }
    const double ops = (double)blocks * p.threads * p.ops_per_thread;
    return ops / ((ms * 1e-3 / 3.0) * sms * clk_hz);
}

}  // namespace

extern "C" int mcubes_unit_rates(double *out, int n_out)
{
    using namespace mcubes;
    if (!out || n_out < 1) return MCUBES_ERR_INVALID_ARG;
    int dev = 0, sms = 0, clk_khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return cuda_status(e);
    const double clk = clk_khz * 1e3;
    const size_t tab_bytes = sizeof(float2) * kAxes * kBins, f32_bytes = sizeof(float) * kAxes * kBins;
    const size_t u32_bytes = sizeof(uint32_t) * kAxes * kBins * 9;
    const size_t u64x1_bytes = sizeof(uint64_t) * kAxes * kBins, u64x4_bytes = 4 * u64x1_bytes;
    const size_t r32_bytes = sizeof(uint32_t) * kAxes * kBins * 8;
    e = cudaFuncSetAttribute(k_atom_u32x8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)u32_bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_red_u64<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)u64x4_bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_red_u32x8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r32_bytes);
    if (e != cudaSuccess) return cuda_status(e);
    float *buf = nullptr;
    e = mc_malloc((void **)&buf, sizeof(float) * (size_t)sms * 4 * kThreads + tab_bytes);
    if (e != cudaSuccess) return cuda_status(e);
    float2 *gtab = reinterpret_cast<float2 *>(buf + (size_t)sms * 4 * kThreads);   // 16-byte aligned
    k_fill_table<<<(kAxes * kBins + 255) / 256, 256>>>(gtab);
    int st = MCUBES_OK;
    double r[kUnitRates] = {};
    const Probe alu{kThreads, 4, 0, 8.0 * kIters};
    r[0] = time_probe(alu, sms, clk, buf, [](unsigned b, int t, size_t m, float *o) { k_ffma<<<b, t, m>>>(o, 1.0000001f, 1e-7f); }, st);
    if (!st)
        r[1] = time_probe(Probe{kThreads, 4, 0, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_dfma<<<b, t, m>>>(o, 1.0000001, 1e-7); }, st);
    if (!st) r[2] = time_probe(alu, sms, clk, buf, [](unsigned b, int t, size_t m, float *o) { k_ex2<<<b, t, m>>>(o); }, st);
    if (!st)
        r[3] = time_probe(Probe{kThreads, 4, 0, 2.0 * (kIters / 4)}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_philox<<<b, t, m>>>(o, 0x12345678u, 0x9abcdef0u); }, st);
    if (!st)
        r[4] = time_probe(Probe{kThreads, 4, tab_bytes, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_gather<<<b, t, m>>>(o, 7u); }, st);
    if (!st)
        r[5] = time_probe(Probe{kThreads, 4, f32_bytes, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_atom_f32<<<b, t, m>>>(o, 7u); }, st);
    if (!st)
        r[6] = time_probe(Probe{4 * kThreads, 1, u32_bytes, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_atom_u32x8<<<b, t, m>>>(o, 7u); }, st);
    if (!st)
        r[7] = time_probe(Probe{4 * kThreads, 1, u64x1_bytes, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_red_u64<1><<<b, t, m>>>(o, 7u); }, st);
    if (!st)
        r[8] = time_probe(Probe{4 * kThreads, 1, u64x4_bytes, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_red_u64<4><<<b, t, m>>>(o, 7u); }, st);
    if (!st)
        r[9] = time_probe(Probe{4 * kThreads, 1, r32_bytes, 1.0 * kIters}, sms, clk, buf,
                          [](unsigned b, int t, size_t m, float *o) { k_red_u32x8<<<b, t, m>>>(o, 7u); }, st);
    if (!st)
        r[10] = time_probe(Probe{kThreads, 4, 0, 1.0 * kIters}, sms, clk, buf,
                           [gtab](unsigned b, int t, size_t m, float *o) { k_gather_l1<false><<<b, t, m>>>(o, gtab, 7u); }, st);
    if (!st)
        r[11] = time_probe(Probe{kThreads, 4, tab_bytes, 1.0 * kIters}, sms, clk, buf,
                           [gtab](unsigned b, int t, size_t m, float *o) { k_gather_l1<true><<<b, t, m>>>(o, gtab, 7u); }, st);
    cudaFree(buf);
    if (st) return st;
    for (int i = 0; i < n_out && i < kUnitRates; ++i) out[i] = r[i];
    return MCUBES_OK;
}
