// The m-Cubes V-Sample kernel (paper Sec. 3.2, Algorithm 2), written for sm_103a.
//
// Work decomposition. A persistent grid (blocks = SMs x resident blocks, N threads). The
// sub-cubes [0, m) are cut into N equal contiguous ranges; thread j owns range
// r = (j perm_mul) mod N, a permutation that scatters a warp's ranges over [0, m). A thread's
// strata digits are decomposed once and then advanced by +1 with carry.
//
// Per sample (Algorithm 2's inner loop):
//   1. Philox4x32-10 draws with counter (t, q, it << 16 | j, job) and key = seed;
//   2. the VEGAS map through the grid staged in shared memory, as (B_k, Delta_k) pairs;
//   3. the integrand, fed coordinate by coordinate;
//   4. the sub-cube sums;
//   5. on adjusting iterations, the bin contributions w^2, added to a block-private
//      shared-memory histogram.
//
// Kernel instances per (d, integrand, precision) by histogram kind HK: 0 for frozen iterations
// (no histogram code at all); 1 for FP64 adjusting iterations (one shared copy); 2 for FP32
// adjusting iterations (a fixed-point histogram, see IntHist).
//
// Per block at the end:
//   - warp-shuffle and shared-memory reduction of the thread sums, then two FP64 global
//     atomics into sums[0..1] (Algorithm 2's AtomicAdd into r);
//   - the private histogram flushed to the global FP64 bin contributions C with one atomic
//     per non-empty bin.
//
// FP64 path: every step in double. The point uses the exact operation sequence of the
// definition, so the bins match a CPU evaluation bit for bit:
//   yn = min((c + u) R, largest double below nd), k = floor(yn), delta = yn - k,
//   x = fma(Delta_k, delta, B_k).
// Its Jacobian factor nd^d is applied once per block.
//
// FP32 path: the same sequence in single precision, with u on 23 bits, so that the bin and
// the point match a CPU single-precision evaluation bit for bit. Then:
//   - the scaled integrand f/F (fast SFU math);
//   - per sub-cube mean and variance from shifted sums (w - w_0) in single precision, summed per
//     thread with compensation and widened to FP64 once per thread;
//   - the bin contributions (w sigma)^2 with sigma = F / |I_prev|, in the fixed-point histogram
//     (IntHist) on adjusting iterations.
// The single-job kernels draw Philox in the hoisted form (philox_prepare / philox_cube /
// philox_draw: launch constants, then per-sub-cube products), the batched kernel in its
// register form; both are bit-identical to philox4x32_10.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "integrands.cuh"

namespace mcubes {

template <bool F32>
struct Prec;
template <>
struct Prec<false> {
    using T = double;
    using T2 = double2;
};
template <>
struct Prec<true> {
    using T = float;
    using T2 = float2;
};

// Shared-memory bytes of one block: the (B, Delta) table and hr copies of the histogram.
template <bool F32>
__host__ __device__ constexpr size_t vsample_smem_bytes(int d, int hr)
{
    return (size_t)d * kNB * (sizeof(typename Prec<F32>::T2) + (size_t)hr * sizeof(typename Prec<F32>::T));
}

// The fixed-point histogram of the FP32 adjusting kernel (HK = 2).
//
// A contribution h (FP32, >= 0) becomes v = h q with q = 2^e a power of two chosen per block, so
// the product is exact. When v < vmax = 2^ih_vmax_exp (at most 2^44) it is rounded to a whole
// number of units (exact from 2^23 units up, within half a unit below) and added to the bin with
// native u32 shared atomics:
//   - the low word to one of R lane-interleaved copies (copy g = lane mod R holds bin e at word
//     e R + g, so only the 32 / R lanes of a copy can meet in a bank). Each add returns the old
//     word; the carry out of old + low word is shifted into a per-sample carry mask;
//   - the high word, plus 1 for each carry, to a single high word per bin, in one branch a sample
//     that runs only when the sample has a high word or a carry (rare: see the scale below).
// Contributions rounding to zero units add nothing. The rest (from vmax up, infinite or NaN) go to
// an FP32 side copy with FP32 shared atomics. The host sets vmax so that a block's samples times
// vmax stays below 2^63: no bin's sum can overflow. The flush adds (low copies + 2^32 high) / q +
// side into the FP64 C.
//
// Why: an FP32 shared atomic costs about four times a u32 one under random bins (it reads the
// word, adds and compares-and-swaps), and the histogram's atomics bound adjusting iterations.
//
// The scale comes from a pilot, each thread's first sample: q puts the pilot's arithmetic mean
// contribution at 2^20 units, or higher where needed to put the block's expected mean bin (its
// samples times that mean over the 500 bins) at 2^30 units (exponent rounded down). The mean, not
// a typical size, is what fixes a bin's sum, so:
//   - at the sizes where speed matters (many samples a bin) the unit is 2^-20 of the mean: the low
//     words wrap, and the high words are touched, about once per 2^12 adds of a mean-sized
//     contribution, and a contribution reaches the high word (2^32 units) or vmax only at 2^12 or
//     2^23 times the mean: by Markov's inequality a small fraction of the samples;
//   - a contribution rounds with an error of half a unit at most, so a block's error in any bin is
//     at most half a unit per contribution against an expected mean bin of 2^30 units or more; a
//     contribution of the mean's size keeps 2^-21 relative precision or better.
// A block whose pilot has no positive finite contribution sends every contribution to the side
// copy.
constexpr int kReplThreads = 1024;
constexpr double kIntHistCentre = 20.0;            // log2 of the pilot's mean contribution, in units (at least)
constexpr double kIntHistBinSum = 30.0;            // log2 of a block's expected mean bin, in units (at least)
template <int D>
__host__ __device__ constexpr size_t int_hist_smem_bytes(int r)
{
    return (size_t)D * kNB * (sizeof(float2) + 4 * (size_t)r + 4 + 4);
}
template <int D>
__host__ __device__ constexpr int int_hist_copies()
{
    return int_hist_smem_bytes<D>(8) + 2048 <= (size_t)227 * 1024 ? 8 : int_hist_smem_bytes<D>(4) + 2048 <= (size_t)227 * 1024 ? 4 : 2;
}

// Shared-memory bytes of one single-job block with histogram kind HK.
template <int D, bool F32, int HK>
__host__ __device__ constexpr size_t single_smem_bytes()
{
    return HK == 2 ? int_hist_smem_bytes<D>(int_hist_copies<D>()) : vsample_smem_bytes<F32>(D, HK);
}

// Shared-window addresses of a block's fixed-point histogram, and its scale.
struct IntHist {
    uint32_t lo;     // R low-word copies: bin e, copy g at word e R + g
    uint32_t hi;     // one high word per bin
    uint32_t side;   // one FP32 word per bin
    float q;         // 2^e: fixed-point units per unit of contribution
    float vmax;      // contributions of vmax units or more go to the side copy
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of two doubles; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *scratch /* 2*32 */)
{
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        scratch[warp] = a;
        scratch[32 + warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        a = lane < nw ? scratch[lane] : 0.0;
        b = lane < nw ? scratch[32 + lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

// Shared-memory accesses by 32-bit shared-window address (FP32 path): the table and histogram
// addresses come straight from the bit pattern of the floored coordinate (below).
__device__ __forceinline__ float2 lds_f32x2(uint32_t a)
{
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void red_add_f32(uint32_t a, float v)
{
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ uint32_t atom_add_u32(uint32_t a, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v));
    return old;
}
// FP64 add into global memory with no returned value (performed by the L2).
__device__ __forceinline__ void red_add_f64_global(double *a, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add_u32(uint32_t a, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v));
}
// mask * 2 + the carry out of old + lo (add with carry-out, then add the mask to itself with the
// carry in): collects a sample's low-word carries, one bit an axis.
__device__ __forceinline__ uint32_t carry_in(uint32_t mask, uint32_t old, uint32_t lo)
{
    uint32_t m;
    asm("{\n\t.reg .u32 s;\n\tadd.cc.u32 s, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}" : "=r"(m) : "r"(old), "r"(lo), "r"(mask));
    return m;
}
// round(v) for a float 0 <= v < 2^44 as a 64-bit integer (lo, hi), with integer operations (a
// 64-bit float conversion would run on the FP64 pipe). Below 2^23, v + 2^23 rounds v to an integer
// (to nearest, ties to even) and its bit pattern is 0x4B000000 + round(v). From 2^23 up, v is the
// integer M 2^s with its 24-bit significand M and s = exponent - 23 in [0, 20].
__device__ __forceinline__ void round_units(float v, uint32_t &lo, uint32_t &hi)
{
    const uint32_t b = __float_as_uint(v);
    const uint32_t M = (b & 0x7FFFFFu) | 0x800000u;
    const uint32_t s = (b >> 23) - 150u;
    const uint32_t small = __float_as_uint(__fadd_rn(v, 8388608.0f)) - 0x4B000000u;
    const bool big = v >= 8388608.0f;
    lo = big ? M << (s & 31u) : small;
    hi = big ? __funnelshift_l(M, 0u, s) : 0u;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One sample's contribution h to the fixed-point histogram (HK = 2) on its d bins; kbb[i] is the bit
// pattern 0x4B000000 + k_i of axis i's floored coordinate, the adj values the shared-window offsets
// that turn it into this lane's low word, the bin's high word and its side word.
template <int D>
__device__ __forceinline__ void fixed_hist_add(const float h, const uint32_t (&kbb)[D], const IntHist &ih,
                                               const uint32_t lo_adj, const uint32_t hi_adj, const uint32_t side_adj)
{
    constexpr int kR = int_hist_copies<D>();
    const float vf = h * ih.q;   // exact: q is a power of two
    if (vf < ih.vmax) {
        uint32_t vlo, vhi;
        round_units(vf, vlo, vhi);
        if ((vlo | vhi) != 0u) {
            uint32_t carries = 0u;   // axis i's carry in bit D - 1 - i
#pragma unroll
            for (int i = 0; i < D; ++i) {
                const uint32_t old = atom_add_u32(kbb[i] * (4u * kR) + (lo_adj + (uint32_t)(i * kNB * 4 * kR)), vlo);
                carries = carry_in(carries, old, vlo);
            }
            if ((carries | vhi) != 0u) {
#pragma unroll
                for (int i = 0; i < D; ++i)
                    red_add_u32(kbb[i] * 4u + (hi_adj + (uint32_t)(i * kNB * 4)), vhi + ((carries >> (D - 1 - i)) & 1u));
            }
        }
    } else if (h != 0.0f) {   // from vmax up, infinite or NaN
#pragma unroll
        for (int i = 0; i < D; ++i) red_add_f32(kbb[i] * 4u + (side_adj + (uint32_t)(i * kNB * 4)), h);
    }
}

// Resident blocks per SM the FP32-eval kernels are compiled for (register budget 65536 /
// (256 x blocks)): for the frozen and batched kernels, as many 256-thread blocks as the shared
// memory of a block with a one-copy histogram allows, at most 4 (64 registers: fewer, with
// spills, measured slower); the fixed-point adjusting kernel runs one 1024-thread block per SM
// (64 registers as well). FP64 kernels are bound by the FP64 pipe and keep the default budget.
#ifndef MCUBES_MAX_MIN_BLOCKS
#define MCUBES_MAX_MIN_BLOCKS 4
#endif
template <int D, bool F32, int HK = 1>
constexpr int min_blocks_per_sm()
{
    if (!F32 || HK == 2) return 1;
    const size_t smem = vsample_smem_bytes<F32>(D, true) + 1024;
    const int fit = (int)((size_t)(227 * 1024) / smem);
    const int b = fit < MCUBES_MAX_MIN_BLOCKS ? fit : MCUBES_MAX_MIN_BLOCKS;
    return b < 1 ? 1 : b;
}

// Per-thread accumulators of one job's sub-cubes.
struct ThreadSums {
    double sI = 0.0, sV = 0.0;      // FP64 path
    float cI = 0.0f, eI = 0.0f;     // FP32 path: Neumaier-compensated sums of the cube means
    float cV = 0.0f, eV = 0.0f;     // ... and of the cube variances (times p (p-1))
};

// Stage a grid into shared memory as (B_k, Delta_k) pairs and clear n_clear 4-byte words of the
// histogram region that follows it. Block-wide.
template <int D, bool F32>
__device__ __forceinline__ void stage_grid(const double *grid, typename Prec<F32>::T2 *tab,
                                           void *hist, int n_clear)
{
    using T = typename Prec<F32>::T;
    using T2 = typename Prec<F32>::T2;
    for (int e = threadIdx.x; e < D * kNB; e += blockDim.x) {
        const int i = e / kNB;
        const int k = e - i * kNB;
        const double b0 = grid[i * (kNB + 1) + k];
        const double b1 = grid[i * (kNB + 1) + k + 1];
        T2 v;
        v.x = (T)b0;
        v.y = (T)(b1 - b0);
        tab[e] = v;
    }
    uint32_t *h = reinterpret_cast<uint32_t *>(hist);
    for (int e = threadIdx.x; e < n_clear; e += blockDim.x) h[e] = 0u;
    __syncthreads();
}

// FP32 histogram scale sigma = F / |I_prev| (1 when unknown).
template <bool F32>
__device__ __forceinline__ float histogram_scale(const VsampleParams &P)
{
    float hsig = 1.0f;
    if (F32 && P.adjust && P.prev != nullptr) {
        const double ip = fabs(P.prev[0] * P.prev_scale);
        if (ip > 0.0 && ip < 1e300 && P.fscale > 0.0) {
            const double s = P.fscale / ip;
            if (s > 1e-30 && s < 1e30) hsig = (float)s;
        }
    }
    return hsig;
}

// Algorithm 2's loop over this thread's sub-cubes [t, t_end): draws, map, integrand, per-cube
// statistics and bin contributions. kGlobalHist routes the contributions straight to the
// job's global C (FP64 atomics) instead of the block's shared histogram; otherwise HK picks the
// block's histogram (0: none, 1: one shared copy `hist`, 2: the fixed-point histogram `ih`).
// kPilot: evaluate only sample q = 0 of sub-cube t and return its contribution (w sigma)^2,
// touching nothing else.
template <int D, int FID, bool F32, bool kGlobalHist, int HK, bool kPre, bool kPilot = false>
__device__ __forceinline__ float sample_cubes(const VsampleParams &P, uint32_t t, const uint32_t t_end,
                                              const typename Prec<F32>::T2 *tab, typename Prec<F32>::T *hist,
                                              const IntHist &ih, const float hsig, ThreadSums &acc)
{
    using T = typename Prec<F32>::T;
    using T2 = typename Prec<F32>::T2;
    static_assert(HK >= 0 && HK <= 2, "histogram kind: 0, 1 or 2");
    static_assert(HK != 2 || F32, "the fixed-point histogram is the FP32 path's");
    static_assert(!kPilot || (F32 && HK == 2), "the pilot serves the fixed-point histogram");
    const bool adjust = (kGlobalHist || HK > 0) && P.adjust != 0;
    constexpr int kR = HK == 2 ? int_hist_copies<D>() : 1;

    // strata digits c_i (axis 0 fastest) and c_i - 1 in the path's precision
    uint32_t dig[D];
    T cm1[D];
    {
        uint32_t rest = t;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            dig[i] = rest % P.g;
            rest /= P.g;
            cm1[i] = (T)dig[i] - T(1);
        }
    }

    const T R = F32 ? (T)P.R32 : (T)P.R;
    const T ycap = F32 ? (T)P.ycap32 : (T)P.ycap;
    const T magic = F32 ? (T)8388608.0f : (T)4503599627370496.0;   // 2^23 / 2^52
    const uint32_t p = P.p;
    const float inv_p32 = (float)P.inv_p;
    // FP32: kb = yn + 2^23 rounded down has bit pattern 0x4B000000 + k, so the byte address of
    // table entry (i, k) is bits(kb) * 8 + tab_adj + i * kNB * 8 (mod 2^32), and the histogram
    // words of bin (i, k) follow the same pattern: one shared copy (HK = 1) at bits(kb) * 4 +
    // hist_adj; fixed point (HK = 2) with this lane's low word at bits(kb) * 4 R + lo_adj and the
    // high and side words at bits(kb) * 4 + hi_adj / side_adj (each plus i times the axis stride).
    constexpr uint32_t kMagicBits = 0x4B000000u;
    const uint32_t tab_adj = smem_addr(tab) - kMagicBits * 8u;
    const uint32_t hist_adj = HK == 1 ? smem_addr(hist) - kMagicBits * 4u : 0u;
    const uint32_t lo_adj = HK == 2 ? ih.lo + 4u * (threadIdx.x & (uint32_t)(kR - 1)) - kMagicBits * (4u * kR) : 0u;
    const uint32_t hi_adj = HK == 2 ? ih.hi - kMagicBits * 4u : 0u;
    const uint32_t side_adj = HK == 2 ? ih.side - kMagicBits * 4u : 0u;
    // global-histogram scale (FP32: (F / sigma)^2; FP64: 1, the contribution already carries nd^d)
    double gscale = 0.0;
    if constexpr (kGlobalHist) {
        if constexpr (F32) {
            const double r = P.fscale / (double)hsig;
            gscale = r * r;
        } else {
            gscale = 1.0;
        }
    }

    // Philox draws: kPre reads the launch's prepared constants (P.ph); otherwise the per-call
    // constants and job ^ key1 are formed here, once, and kept in registers
    constexpr int kDimsPerCall = F32 ? 4 : 2;
    constexpr int kCalls = (D + kDimsPerCall - 1) / kDimsPerCall;
    static_assert(kCalls <= kPhiloxPreWords, "the prepared constants cover every draw word of a sample");
    uint32_t pa[kCalls], pbk[kCalls];
    uint32_t job_key1 = 0u;
    if constexpr (!kPre) {
#pragma unroll
        for (int j = 0; j < kCalls; ++j) philox_draw_consts(P.key0, P.ctr2_hi, j, pa[j], pbk[j]);
        job_key1 = P.job ^ P.key1;
    }

    for (; t < t_end; ++t) {
        if (!mc_check(P.chk, t, P.m, 3)) break;
        T S1 = T(0), S2 = T(0), w0 = T(0);   // FP64: plain sums; FP32: w0 and shifted sums
        PhiloxCube cube;
        if constexpr (kPre) {
            cube = philox_cube(t, P.ph);
        } else {
            cube = philox_cube_k(t, job_key1);
        }

        for (uint32_t q = 0; q < p; ++q) {
            Integrand64<FID, D> f64;
            Integrand32<FID, D> f32;
            T J = T(1);
            int kofs[D];        // bin index i nd + k (FP64 path, global histogram)
            uint32_t kbb[D];    // bit pattern of yn + 2^23 rounded down: 0x4B000000 + k (FP32 path)

#pragma unroll
            for (int j = 0; j < kCalls; ++j) {
                Words4 r;
                if constexpr (kPre) {
                    r = philox_draw(q, j, cube, P.ph);
                } else {
                    r = philox_draw_k(q, pa[j], pbk[j], cube, P.key0, P.key1);
                }
                const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int h = 0; h < kDimsPerCall; ++h) {
                    const int i = j * kDimsPerCall + h;
                    if (i < D) {
                        // f = 1 + u exactly; (c - 1) + f rounds like c + u
                        T f;
                        if constexpr (F32) {
                            f = __uint_as_float((wv[h] & 0x7FFFFFu) | 0x3F800000u);
                        } else {
                            f = __hiloint2double((int)((wv[2 * h] & 0xFFFFFu) | 0x3FF00000u), (int)wv[2 * h + 1]);
                        }
                        T yn;
                        if constexpr (F32) {
                            yn = __fmul_rn(__fadd_rn(cm1[i], f), R);
                            yn = fminf(yn, ycap);
                        } else {
                            // the cap min(yn, largest double below nd) is applied below, on the rare
                            // floor >= nd (yn < nd already lies at or below the cap)
                            yn = __dmul_rn(__dadd_rn(cm1[i], f), R);
                        }
                        // floor(yn) for 0 <= yn < 2^23 (2^52): add the magic number rounding down
                        T kb;
                        T2 bw;
                        if constexpr (F32) {
                            kb = __fadd_rd(yn, magic);
                            uint32_t kbits = __float_as_uint(kb);
                            if (!mc_check(P.chk, (long long)kbits - (long long)kMagicBits, kNB, 1)) kbits = kMagicBits;
                            bw = lds_f32x2(kbits * 8u + (tab_adj + (uint32_t)(i * kNB * 8)));
                            if constexpr (kGlobalHist) {
                                kofs[i] = i * kNB + (int)(kbits - kMagicBits);
                            } else {
                                kbb[i] = kbits;
                            }
                            kb = __fsub_rn(kb, magic);
                        } else {
                            kb = __dadd_rd(yn, magic);
                            int k = __double2loint(kb);
                            if (k >= kNB) {   // yn rounded up to nd: cap it, as min(yn, ycap) would
                                yn = ycap;
                                kb = __dadd_rd(yn, magic);
                                k = __double2loint(kb);
                            }
                            if (!mc_check(P.chk, k, kNB, 1)) k = 0;
                            bw = tab[i * kNB + k];
                            kofs[i] = i * kNB + k;
                            kb = __dsub_rn(kb, magic);
                        }
                        const T delta = yn - kb;     // exact
                        T x;
                        if constexpr (F32) {
                            x = __fmaf_rn(bw.y, delta, bw.x);
                            f32.add(i, x, P.ip);
                        } else {
                            x = __fma_rn(bw.y, delta, bw.x);
                            f64.add(i, x, P.ip);
                        }
                        J *= bw.y;
                        if constexpr (F32) {
                            // keep J near 1: fold nd^4 in after every fourth axis
                            if ((i & 3) == 3) J *= 6.25e10f;
                        }
                    }
                }
            }
            T w;
            if constexpr (F32) {
                constexpr int rem = D & 3;
                if (rem == 1) J *= 500.0f;
                if (rem == 2) J *= 250000.0f;
                if (rem == 3) J *= 125000000.0f;
                w = f32.finish(P.ip) * J;
            } else {
                w = f64.finish(P.ip) * J;   // Jacobian without nd^d (applied per block)
            }

            if constexpr (kPilot) {
                const float ws = w * hsig;
                return ws * ws;
            }
            if constexpr (F32) {
                if (q == 0) {
                    w0 = w;
                } else {
                    const float dv = w - w0;
                    S1 += dv;
                    S2 = fmaf(dv, dv, S2);
                }
            } else {
                S1 += w;
                S2 = fma(w, w, S2);
            }

            if (adjust) {
                T h;
                if constexpr (F32) {
                    const float ws = w * hsig;
                    h = ws * ws;
                } else {
                    // the full weight (with the Jacobian's nd^d) squared: the same range as the
                    // contribution itself, so it underflows only where the contribution does
                    const double wf = w * P.fscale;
                    h = wf * wf;
                }
                if constexpr (kGlobalHist) {
                    const double hg = (double)h * gscale;
#pragma unroll
                    for (int i = 0; i < D; ++i)
                        if (mc_check(P.chk, kofs[i], D * kNB, 2)) atomicAdd(&P.C[kofs[i]], hg);
                } else if constexpr (HK == 1) {
                    if constexpr (F32) {
#pragma unroll
                        for (int i = 0; i < D; ++i) red_add_f32(kbb[i] * 4u + (hist_adj + (uint32_t)(i * kNB * 4)), h);
                    } else {
#pragma unroll
                        for (int i = 0; i < D; ++i) atomicAdd(&hist[kofs[i]], h);
                    }
                } else if constexpr (HK == 2) {
                    fixed_hist_add<D>(h, kbb, ih, lo_adj, hi_adj, side_adj);
                }
            }
        }

        // per sub-cube mean and variance (Algorithm 2 UpdateVariance)
        const bool probe_this = P.probe != nullptr && (t & P.probe_mask) == 0 &&
                                mc_check(P.chk, t >> P.probe_shift, (long long)(P.m >> P.probe_shift) + 1, 4);
        if constexpr (F32) {
            // Single precision on the shifted sums: mean = w0 + D1/p, p(p-1) V = D2 - D1^2/p.
            // The shift keeps D2 - D1^2/p free of the cancellation of S2 - S1^2/p. The
            // per-thread sums are compensated (Neumaier) and widened to FP64 once per thread.
            const float mean = fmaf(S1, inv_p32, w0);
            float var = fmaf(-S1 * inv_p32, S1, S2);
            var = fmaxf(var, 0.0f);
            {
                const float tI = acc.cI + mean;
                acc.eI += (fabsf(acc.cI) >= fabsf(mean)) ? ((acc.cI - tI) + mean) : ((mean - tI) + acc.cI);
                acc.cI = tI;
                const float tV = acc.cV + var;
                acc.eV += (acc.cV >= var) ? ((acc.cV - tV) + var) : ((var - tV) + acc.cV);
                acc.cV = tV;
            }
            if (probe_this) {   // probe values on the final scale (fscale = F)
                P.probe[2 * (size_t)(t >> P.probe_shift)] = (double)mean * P.fscale;
                P.probe[2 * (size_t)(t >> P.probe_shift) + 1] = (double)var * P.inv_pp1 * P.fscale * P.fscale;
            }
        } else {
            const double It = S1 * P.inv_p;
            double Vt = fma(-S1 * P.inv_p, S1, S2);
            Vt = Vt > 0.0 ? Vt : 0.0;
            acc.sI += It;
            acc.sV += Vt;
            if (probe_this) {   // probe values on the final scale (fscale = nd^d)
                P.probe[2 * (size_t)(t >> P.probe_shift)] = It * P.fscale;
                P.probe[2 * (size_t)(t >> P.probe_shift) + 1] = Vt * P.inv_pp1 * P.fscale * P.fscale;
            }
        }

        // advance the strata digits to sub-cube t + 1
        bool carry = true;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if (carry) {
                if (++dig[i] < P.g) {
                    cm1[i] += T(1);
                    carry = false;
                } else {
                    dig[i] = 0;
                    cm1[i] = T(-1);
                }
            }
        }
    }
    return 0.0f;
}

// Block reduction of the thread sums, two FP64 global atomics into P.sums (Algorithm 2,
// AtomicAdd into r), then the flush of the block's histogram into P.C: one shared copy (HK = 1),
// or the fixed-point histogram (HK = 2; per bin, (low copies + 2^32 high) / q + side). Block-wide;
// leaves the histogram free for reuse (ends with a barrier).
template <int D, bool F32, int HK>
__device__ __forceinline__ void finish_block(const VsampleParams &P, ThreadSums &acc,
                                             typename Prec<F32>::T *hist, const IntHist &ih, bool flush_hist,
                                             float hsig, double *red_scratch)
{
    using T = typename Prec<F32>::T;
    double sI = acc.sI, sV = acc.sV;
    if constexpr (F32) {
        sI = (double)acc.cI + (double)acc.eI;
        sV = (double)acc.cV + (double)acc.eV;
    }
    block_sum2(sI, sV, red_scratch);
    if (threadIdx.x == 0) {
        atomicAdd(&P.sums[0], sI * P.fscale);
        atomicAdd(&P.sums[1], sV * P.inv_pp1 * P.fscale * P.fscale);
    }
    if (HK > 0 && flush_hist) {
        __syncthreads();
        double cscale;
        if constexpr (F32) {
            const double r = P.fscale / (double)hsig;
            cscale = r * r;
        } else {
            cscale = 1.0;   // the block's contributions already carry nd^(2d)
        }
        if constexpr (HK == 2) {
            constexpr int kR = int_hist_copies<D>();
            const uint32_t *lo = reinterpret_cast<const uint32_t *>(hist);
            const uint32_t *hi = lo + (size_t)D * kNB * kR;
            const float *side = reinterpret_cast<const float *>(hi + (size_t)D * kNB);
            const double inv_q = 1.0 / (double)ih.q;
            for (int e = threadIdx.x; e < D * kNB; e += blockDim.x) {
                unsigned long long sum = (unsigned long long)hi[e] << 32;
                if constexpr (kR >= 4) {
                    // the copies of bin e are kR consecutive words, 16-byte aligned
                    const uint4 *q4 = reinterpret_cast<const uint4 *>(lo + (size_t)e * kR);
#pragma unroll
                    for (int c = 0; c < kR / 4; ++c) {
                        const uint4 b = q4[c];
                        sum += (unsigned long long)b.x + b.y + (unsigned long long)b.z + b.w;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < kR; ++c) sum += lo[(size_t)e * kR + c];
                }
                double v = (double)side[e];
                if (sum != 0ull) v += (double)sum * inv_q;
                if (v != 0.0) atomicAdd(&P.C[e], v * cscale);
            }
        } else {
            for (int e = threadIdx.x; e < D * kNB; e += blockDim.x) {
                const T v = hist[e];
                if (v != T(0)) atomicAdd(&P.C[e], (double)v * cscale);
            }
        }
    }
    __syncthreads();
}

// One job, whole grid of persistent blocks. HK = 0: frozen iteration; HK = 1: FP64 adjusting
// iteration; HK = 2: FP32 adjusting iteration with the fixed-point histogram, one 1024-thread
// block per SM.
template <int D, int FID, bool F32, int HK>
__global__ void __launch_bounds__((HK == 2 ? kReplThreads : kMaxBlockThreads), (min_blocks_per_sm<D, F32, HK>()))
    vsample_kernel(const VsampleParams P)
{
    using T = typename Prec<F32>::T;
    using T2 = typename Prec<F32>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *tab = reinterpret_cast<T2 *>(smem_raw);
    T *hist = reinterpret_cast<T *>(smem_raw + (size_t)D * kNB * sizeof(T2));
    __shared__ double red_scratch[64];
    __shared__ float pilot_q, pilot_vmax;

    constexpr int kR = HK == 2 ? int_hist_copies<D>() : 1;
    const bool adjust = HK > 0 && P.adjust != 0;
    // histogram words: one copy (HK = 1, T-sized), or kR low copies + high + side (HK = 2)
    const int n_clear = !adjust ? 0 : HK == 2 ? D * kNB * (kR + 2) : D * kNB * (int)(sizeof(T) / 4);
    stage_grid<D, F32>(P.grid, tab, hist, n_clear);

    // This thread's sub-cube range. Range r = (gtid * P.perm_mul) mod N is a permutation of
    // the N threads (perm_mul is odd and coprime with N): the 32 lanes of a warp start in
    // scattered parts of [0, m), so their strata differ on every axis and their bins spread
    // over the whole histogram instead of piling into one stratum's window.
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t rng = (gtid * (uint64_t)P.perm_mul) % nthreads;
    const uint32_t t = (uint32_t)((rng * P.m) / nthreads);
    const uint32_t t_end = (uint32_t)(((rng + 1) * P.m) / nthreads);

    const float hsig = histogram_scale<F32>(P);
    ThreadSums acc;
    IntHist ih{0u, 0u, 0u, 0.0f, 0.0f};
    if constexpr (HK == 2) {
        ih.lo = smem_addr(hist);
        ih.hi = ih.lo + 4u * (uint32_t)(D * kNB * kR);
        ih.side = ih.hi + 4u * (uint32_t)(D * kNB);
        ih.vmax = ldexpf(1.0f, P.ih_vmax_exp);
        if (adjust) {
            // pilot: the threads' first contributions (the sum of the finite ones and their count),
            // and the block's sample count
            double hsum = 0.0, nfin = 0.0;
            if (t < t_end) {
                const float hp = sample_cubes<D, FID, F32, false, HK, true, true>(P, t, t + 1, tab, hist, ih, hsig, acc);
                if (hp <= 3.0e38f) {   // finite (NaN compares false)
                    hsum = (double)hp;
                    nfin = 1.0;
                }
            }
            block_sum2(hsum, nfin, red_scratch);
            double nsamp = (double)(t_end - t) * (double)P.p, unused = 0.0;
            __syncthreads();   // red_scratch is reused
            block_sum2(nsamp, unused, red_scratch);
            if (threadIdx.x == 0) {
                float q = 1.0f, vmax = 0.0f;   // no positive pilot contribution: all to the side copy
                if (hsum > 0.0 && nfin > 0.0 && nsamp > 0.0) {
                    // the pilot's mean at 2^kIntHistCentre units or more, and the block's expected
                    // mean bin (samples x pilot mean / kNB) at 2^kIntHistBinSum units or more
                    const double lg = fmax(kIntHistCentre, kIntHistBinSum + log2((double)kNB / nsamp));
                    const double e = floor(lg - log2(hsum / nfin));
                    q = ldexpf(1.0f, (int)fmin(fmax(e, -120.0), 120.0));
                    vmax = ih.vmax;
                }
                pilot_q = q;
                pilot_vmax = vmax;
            }
            __syncthreads();
            ih.q = pilot_q;
            ih.vmax = pilot_vmax;
        }
    }
    sample_cubes<D, FID, F32, false, HK, true>(P, t, t_end, tab, hist, ih, hsig, acc);
    finish_block<D, F32, HK>(P, acc, hist, ih, adjust, hsig, red_scratch);
}

// ------------------------------------------------------------------------------ batches
// Many independent integrations in one launch. The host cuts every job of one (d, family)
// class into tiles of consecutive sub-cubes. Block b takes the contiguous tile range
// [b n / B, (b+1) n / B), so it switches job only at job boundaries. On each switch it flushes
// the finished job's sums and histogram and stages the next job's grid.
struct BatchJob {
    VsampleParams P;            // per-job constants (grid, C, sums, prev are set per iteration)
    const double *grid[2];      // ping-pong grids
    double *C;                  // d x 500 bin contributions
    double *sums;               // 2 x itmax per-iteration sums
};

struct BatchTile {
    uint32_t job, c0, c1, pad;
};

// The batched kernel keeps one shared copy of the histogram (or none, with kGlobalHist).
__device__ constexpr IntHist kNoIntHist{0u, 0u, 0u, 0.0f, 0.0f};

template <int D, int FID, bool F32, bool kGlobalHist>
__global__ void __launch_bounds__(kMaxBlockThreads, (min_blocks_per_sm<D, F32>()))
    vsample_batch_kernel(const BatchJob *__restrict__ jobs, const BatchTile *__restrict__ tiles, int n_tiles,
                         int iteration, int parity, int adjust, uint32_t perm_mul)
{
    using T = typename Prec<F32>::T;
    using T2 = typename Prec<F32>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *tab = reinterpret_cast<T2 *>(smem_raw);
    T *hist = reinterpret_cast<T *>(smem_raw + (size_t)D * kNB * sizeof(T2));
    __shared__ double red_scratch[64];

    const int tb = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
    const int te = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
    const bool shared_hist = adjust && !kGlobalHist;
    // thread order inside a tile, permuted as in the single-job kernel
    const uint32_t r = (uint32_t)(((uint64_t)threadIdx.x * perm_mul) % blockDim.x);

    int cur = -1;
    VsampleParams P;
    float hsig = 1.0f;
    ThreadSums acc;
    for (int ti = tb; ti < te; ++ti) {
        const BatchTile tile = tiles[ti];
        if ((int)tile.job != cur) {
            if (cur >= 0) {
                finish_block<D, F32, 1>(P, acc, hist, kNoIntHist, shared_hist, hsig, red_scratch);
                acc = ThreadSums();
            }
            cur = (int)tile.job;
            const BatchJob &J = jobs[cur];
            P = J.P;
            P.grid = J.grid[parity];
            P.C = J.C;
            P.sums = J.sums + 2 * iteration;
            P.prev = iteration > 0 ? J.sums + 2 * (iteration - 1) : nullptr;
            P.prev_scale = 1.0 / (double)P.m;
            P.ctr2_hi = (uint32_t)iteration << 16;
            P.adjust = adjust;
            P.probe = nullptr;
            hsig = histogram_scale<F32>(P);
            stage_grid<D, F32>(P.grid, tab, hist, shared_hist ? D * kNB * (int)(sizeof(T) / 4) : 0);
        }
        if (!mc_check(P.chk, (long long)tile.c1 - 1, P.m, 5) || !mc_check(P.chk, tile.c0, (long long)tile.c1, 5)) continue;
        const uint32_t n = tile.c1 - tile.c0;
        const uint32_t t = tile.c0 + (uint32_t)(((uint64_t)r * n) / blockDim.x);
        const uint32_t t_end = tile.c0 + (uint32_t)(((uint64_t)(r + 1) * n) / blockDim.x);
        sample_cubes<D, FID, F32, kGlobalHist, 1, false>(P, t, t_end, tab, hist, kNoIntHist, hsig, acc);
    }
    if (cur >= 0) finish_block<D, F32, 1>(P, acc, hist, kNoIntHist, shared_hist, hsig, red_scratch);
}

}  // namespace mcubes
