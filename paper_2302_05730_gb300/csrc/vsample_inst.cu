// One (precision, integrand) slice of the V-Sample kernel instances, for d = 1..16. Compiled
// once per slice with -DMCUBES_F32=0|1 -DMCUBES_FID=0..7 so the instances build in parallel.
#include <atomic>
#include <cmath>
#include <numeric>

#include "internal.h"
#include "vsample.cuh"
#include "vsample64.cuh"

#ifndef MCUBES_F32
#error "MCUBES_F32 must be defined"
#endif
#ifndef MCUBES_FID
#error "MCUBES_FID must be defined"
#endif
#ifndef MCUBES_PART
#define MCUBES_PART 0   // 0: single-job kernels, 1: batched kernels
#endif

#if MCUBES_F32
#define MCUBES_PREC f32
#else
#define MCUBES_PREC f64
#endif
#define MCUBES_CAT2(a, b, c) launch_vsample_##a##_##b
#define MCUBES_CAT(a, b) MCUBES_CAT2(a, b, 0)
#define MCUBES_LAUNCHER MCUBES_CAT(MCUBES_PREC, MCUBES_FID)
#define MCUBES_BCAT2(a, b) launch_vsample_batch_##a##_##b
#define MCUBES_BCAT(a, b) MCUBES_BCAT2(a, b)
#define MCUBES_BATCH_LAUNCHER MCUBES_BCAT(MCUBES_PREC, MCUBES_FID)

namespace mcubes {
namespace {

constexpr bool kF32 = MCUBES_F32 != 0;
constexpr int kFid = MCUBES_FID;

// Per-instance launch facts, filled on a device's first use of the instance (benign race: every
// writer stores the same values for the same device). The shared-memory attribute is a per-device
// setting, so the facts are kept per device.
constexpr int kMaxDevices = 64;
struct InstanceInfo {
    std::atomic<int> ready[kMaxDevices] = {};
    int occ[kMaxDevices];   // resident blocks per SM at the instance's default block size
};

// The kernel's shared-memory attribute and its residency at `threads` on the current device, set and
// measured once per device.
template <typename Kern>
int instance_occupancy(InstanceInfo &info, Kern kern, int threads, size_t smem, int &occ)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
    if (!info.ready[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
        if (e != cudaSuccess) return (int)e;
        info.occ[dev] = nb > 0 ? nb : 1;
        info.ready[dev].store(1, std::memory_order_release);
    }
    occ = info.occ[dev];
    return (int)cudaSuccess;
}

// Persistent-grid shape and per-launch constants shared by the single-job kernels: blocks, the range
// permutation multiplier, the fixed-point histogram's range and the prepared Philox constants.
inline uint64_t single_launch_shape(VsampleParams &Q, const VsampleParams &P, const LaunchReq &req, int threads,
                                    int bps)
{
    uint64_t blocks = (uint64_t)req.num_sms * (uint64_t)bps;
    // at least ~4 sub-cubes per thread so the per-block grid staging stays cheap
    const uint64_t want = ((uint64_t)P.m + (uint64_t)threads * 4 - 1) / ((uint64_t)threads * 4);
    if (want < blocks) blocks = want;
    if (blocks < 1) blocks = 1;
    // range permutation multiplier: near N / 32 * golden ratio, odd, coprime with N
    Q = P;
    const uint64_t n = blocks * (uint64_t)threads;
    uint64_t mul = (uint64_t)((double)n * 0.6180339887498949) | 1u;
    while (std::gcd(mul, n) != 1) mul += 2;
    Q.perm_mul = (uint32_t)(mul % n == 0 ? 1 : mul % n);
    // fixed-point histogram range: a block adds at most (its threads x the longest thread range x
    // p) contributions to one bin; each below 2^e keeps the 64-bit sum below 2^63
    const uint64_t spb = (((uint64_t)P.m + n - 1) / n) * (uint64_t)P.p * (uint64_t)threads;
    int lg = 0;
    while ((1ull << lg) < spb) ++lg;
    Q.ih_vmax_exp = 63 - lg < 44 ? 63 - lg : 44;
    philox_prepare(Q.ph, Q.key0, Q.key1, Q.ctr2_hi, Q.job);
    return blocks;
}

// One single-job launch of vsample_kernel<D, fid, precision, HK>: a persistent grid of
// num_sms x resident blocks (or the requested blocks per SM).
template <int D, int HK>
int launch_hr(const VsampleParams &P, const LaunchReq &req, cudaStream_t s)
{
    static InstanceInfo info;
    auto kern = vsample_kernel<D, kFid, kF32, HK>;
    constexpr bool kRepl = HK == 2;   // one 1024-thread block per SM
    constexpr int kDefThreads = kRepl ? kReplThreads : kMaxBlockThreads;
    constexpr size_t smem = single_smem_bytes<D, kF32, HK>();
    int occ = 1;
    int e = instance_occupancy(info, kern, kDefThreads, smem, occ);
    if (e != (int)cudaSuccess) return e;
    const int threads = req.user_threads ? req.threads : kDefThreads;
    int bps = req.blocks_per_sm;
    if (bps <= 0) {
        bps = occ;
        // occupancy was computed for the default block size; smaller blocks fit proportionally
        // more, up to the shared memory (the fixed-point histogram: one block per SM whatever its size)
        if (!kRepl && threads < kDefThreads) bps = bps * (kDefThreads / threads);
    }
    VsampleParams Q;
    const uint64_t blocks = single_launch_shape(Q, P, req, threads, bps);
    kern<<<(unsigned)blocks, threads, smem, s>>>(Q);
    return (int)cudaGetLastError();
}

template <int D, int HK>
int launch_fast64(const VsampleParams &P, const LaunchReq &req, cudaStream_t s, bool &launched)
{
    launched = false;
    if constexpr (kF32 || !Fast64<kFid>::kOn) {
        (void)P; (void)req; (void)s;
        return (int)cudaSuccess;
    } else {
        VsampleParams F = P;
        if (!fast64_fold(kFid, F, D)) return (int)cudaSuccess;
        static InstanceInfo info;
        auto kern = vsample_fast64_kernel<D, kFid, HK>;
        constexpr size_t smem = fast64_smem_bytes<D, kFid, HK>();
        if (smem > (size_t)227 * 1024) return (int)cudaSuccess;
        int occ = 1;
        constexpr int kThreads = fast64_threads(D);
        int e = instance_occupancy(info, kern, kThreads, smem, occ);
        if (e != (int)cudaSuccess) return e;
        const int threads = req.user_threads ? req.threads : kThreads;
        int bps = req.blocks_per_sm;
        if (bps <= 0) {
            bps = occ;
            if (threads < kThreads) bps = bps * (kThreads / threads);
        }
        VsampleParams Q;
        const uint64_t blocks = single_launch_shape(Q, F, req, threads, bps);
        kern<<<(unsigned)blocks, threads, smem, s>>>(Q);
        launched = true;
        return (int)cudaGetLastError();
    }
}

// Frozen iterations take the histogram-free instance; adjusting ones the FP32 kernel with the
// fixed-point histogram, or an FP64 kernel: the fast one for the Genz families (half the axes on the
// L2, half in lane-interleaved shared copies), else the plain one with one shared copy.
template <int D>
int launch_d(const VsampleParams &P, const LaunchReq &req, cudaStream_t s)
{
    if (!kF32 && !req.plain64) {
        bool launched = false;
        const int e = P.adjust == 0 ? launch_fast64<D, 0>(P, req, s, launched) : launch_fast64<D, 1>(P, req, s, launched);
        if (launched || e != (int)cudaSuccess) return e;
    }
    if (P.adjust == 0) return launch_hr<D, 0>(P, req, s);
    return launch_hr<D, kF32 ? 2 : 1>(P, req, s);
}

#if MCUBES_PART == 1
struct BatchInstanceInfo {
    std::atomic<int> ready[kMaxDevices] = {};
    int occ[kMaxDevices][2];   // resident blocks per SM at 256 threads, [shared histogram]
};

template <int D, bool kGlobalHist>
int launch_batch_d(const BatchJob *jobs, const BatchTile *tiles, int n_tiles, int iteration, int parity,
                   int adjust, const LaunchReq &req, cudaStream_t s)
{
    static BatchInstanceInfo info;
    auto kern = vsample_batch_kernel<D, kFid, kF32, kGlobalHist>;
    const bool shared_hist = adjust && !kGlobalHist;
    const size_t smem = vsample_smem_bytes<kF32>(D, shared_hist ? 1 : 0);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
    if (!info.ready[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)vsample_smem_bytes<kF32>(D, 1));
        if (e != cudaSuccess) return (int)e;
        for (int a = 0; a < 2; ++a) {
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kMaxBlockThreads,
                                                              vsample_smem_bytes<kF32>(D, a));
            if (e != cudaSuccess) return (int)e;
            info.occ[dev][a] = nb > 0 ? nb : 1;
        }
        info.ready[dev].store(1, std::memory_order_release);
    }
    const int threads = req.threads;
    int bps = req.blocks_per_sm;
    if (bps <= 0) {
        bps = info.occ[dev][shared_hist ? 1 : 0];
        if (threads < kMaxBlockThreads) bps = bps * (kMaxBlockThreads / threads);
    }
    int blocks = req.num_sms * bps;
    if (blocks > n_tiles) blocks = n_tiles;
    if (blocks < 1) return (int)cudaSuccess;
    const uint32_t perm_mul = ((uint32_t)((double)threads * 0.6180339887498949)) | 1u;
    kern<<<blocks, threads, smem, s>>>(jobs, tiles, n_tiles, iteration, parity, adjust, perm_mul);
    return (int)cudaGetLastError();
}

// The batched fast FP64 kernel (vsample64.cuh) of one (d, family) class whose jobs all carry the fold.
template <int D>
int launch_batch_fast_d(const BatchJob *jobs, const BatchTile *tiles, int n_tiles, int iteration, int parity,
                        int adjust, const LaunchReq &req, cudaStream_t s)
{
    if constexpr (kF32 || !Fast64<kFid>::kOn) {
        (void)jobs; (void)tiles; (void)n_tiles; (void)iteration; (void)parity; (void)adjust; (void)req; (void)s;
        return (int)cudaErrorInvalidValue;
    } else {
        static InstanceInfo info;
        auto kern = vsample_batch_fast64_kernel<D, kFid>;
        constexpr size_t smem = fast64_batch_smem_bytes<D, kFid>();
        if (smem > (size_t)227 * 1024) return (int)cudaErrorInvalidValue;
        int occ = 1;
        const int e = instance_occupancy(info, kern, kMaxBlockThreads, smem, occ);
        if (e != (int)cudaSuccess) return e;
        const int threads = req.threads;
        int bps = req.blocks_per_sm;
        if (bps <= 0) {
            bps = occ;
            if (threads < kMaxBlockThreads) bps = bps * (kMaxBlockThreads / threads);
        }
        int blocks = req.num_sms * bps;
        if (blocks > n_tiles) blocks = n_tiles;
        if (blocks < 1) return (int)cudaSuccess;
        const uint32_t perm_mul = ((uint32_t)((double)threads * 0.6180339887498949)) | 1u;
        kern<<<blocks, threads, smem, s>>>(jobs, tiles, n_tiles, iteration, parity, adjust, perm_mul);
        return (int)cudaGetLastError();
    }
}

int launch_batch_fast(int d, const BatchJob *jobs, const BatchTile *tiles, int n_tiles, int iteration, int parity,
                      int adjust, const LaunchReq &req, cudaStream_t s)
{
    switch (d) {
#define MCUBES_FAST_CASE(DD) \
    case DD: return launch_batch_fast_d<DD>(jobs, tiles, n_tiles, iteration, parity, adjust, req, s);
    MCUBES_FAST_CASE(1) MCUBES_FAST_CASE(2) MCUBES_FAST_CASE(3) MCUBES_FAST_CASE(4)
    MCUBES_FAST_CASE(5) MCUBES_FAST_CASE(6) MCUBES_FAST_CASE(7) MCUBES_FAST_CASE(8)
    MCUBES_FAST_CASE(9) MCUBES_FAST_CASE(10) MCUBES_FAST_CASE(11) MCUBES_FAST_CASE(12)
    MCUBES_FAST_CASE(13) MCUBES_FAST_CASE(14) MCUBES_FAST_CASE(15) MCUBES_FAST_CASE(16)
#undef MCUBES_FAST_CASE
    default: return (int)cudaErrorInvalidValue;
    }
}

template <bool kGlobalHist>
int launch_batch(int d, const BatchJob *jobs, const BatchTile *tiles, int n_tiles, int iteration, int parity,
                 int adjust, const LaunchReq &req, cudaStream_t s)
{
    switch (d) {
#define MCUBES_BATCH_CASE(DD) \
    case DD: return launch_batch_d<DD, kGlobalHist>(jobs, tiles, n_tiles, iteration, parity, adjust, req, s);
    MCUBES_BATCH_CASE(1) MCUBES_BATCH_CASE(2) MCUBES_BATCH_CASE(3) MCUBES_BATCH_CASE(4)
    MCUBES_BATCH_CASE(5) MCUBES_BATCH_CASE(6) MCUBES_BATCH_CASE(7) MCUBES_BATCH_CASE(8)
    MCUBES_BATCH_CASE(9) MCUBES_BATCH_CASE(10) MCUBES_BATCH_CASE(11) MCUBES_BATCH_CASE(12)
    MCUBES_BATCH_CASE(13) MCUBES_BATCH_CASE(14) MCUBES_BATCH_CASE(15) MCUBES_BATCH_CASE(16)
#undef MCUBES_BATCH_CASE
    default: return (int)cudaErrorInvalidValue;
    }
}

#endif
}  // namespace

#if MCUBES_PART == 1
int MCUBES_BATCH_LAUNCHER(int d, const BatchJob *jobs, const BatchTile *tiles, int n_tiles, int iteration,
                          int parity, int adjust, int hist_mode, const LaunchReq &req, cudaStream_t s)
{
    if (hist_mode == 2) return launch_batch_fast(d, jobs, tiles, n_tiles, iteration, parity, adjust, req, s);
    return hist_mode == 1 ? launch_batch<true>(d, jobs, tiles, n_tiles, iteration, parity, adjust, req, s)
                          : launch_batch<false>(d, jobs, tiles, n_tiles, iteration, parity, adjust, req, s);
}
#else
int MCUBES_LAUNCHER(int d, const VsampleParams &P, const LaunchReq &req, cudaStream_t s)
{
    switch (d) {
    case 1: return launch_d<1>(P, req, s);
    case 2: return launch_d<2>(P, req, s);
    case 3: return launch_d<3>(P, req, s);
    case 4: return launch_d<4>(P, req, s);
    case 5: return launch_d<5>(P, req, s);
    case 6: return launch_d<6>(P, req, s);
    case 7: return launch_d<7>(P, req, s);
    case 8: return launch_d<8>(P, req, s);
    case 9: return launch_d<9>(P, req, s);
    case 10: return launch_d<10>(P, req, s);
    case 11: return launch_d<11>(P, req, s);
    case 12: return launch_d<12>(P, req, s);
    case 13: return launch_d<13>(P, req, s);
    case 14: return launch_d<14>(P, req, s);
    case 15: return launch_d<15>(P, req, s);
    case 16: return launch_d<16>(P, req, s);
    default: return (int)cudaErrorInvalidValue;
    }
}

#endif

}  // namespace mcubes
