// The FP64 V-Sample kernel for the six Genz families (paper Sec. 3.2, Algorithm 2; Eq. 1-6),
// arranged for GB300's FP64 pipe, which issues about 1/64 of the FP32 rate. Each FP64 operation
// the definition does not need is moved off that pipe, while every step keeps FP64 accuracy and
// the bin index stays bit-identical to the definition's:
//   - c + u rounded to FP64 (nearest even, as an FP64 addition rounds) is built from the integers
//     c 2^52 + bits, and yn = (c + u) R from the 106-bit integer product of the two significands,
//     rounded to nearest even as the FP64 multiply rounds it: both with integer operations, and yn
//     bit-identical to the definition's (the bin depends on its rounding);
//   - the bin k = floor(yn) and the offset in the bin come from the bits of yn with integer
//     operations: for yn >= 1, G = 1 + (yn - k) is exact and is built by shifting the fraction
//     bits of yn under the exponent of 1; for yn < 1 (bin 0) G is 1 + yn cut to 52 fraction bits
//     (an error below 2^-52 of the bin's width);
//   - the family's per-axis linear term is folded into the block's grid table: per bin
//     P_k = a Delta_k and Q_k = (a (B_k - u) or a B_k) - P_k, so that a (x - u) (or a x) is one
//     fma(P_k, G, Q_k) -- the same value as the definition's up to the rounding of the table
//     entries (a few ulps of a Delta_k and a B_k); for the families that only need the sum
//     sum_i a_i x_i (oscillatory, corner peak, discontinuous) the constant parts Q_k are held as
//     64-bit fixed-point integers and summed exactly with integer additions, so each axis costs
//     one FP64 fma into the sum;
//   - the Jacobian prod_i nd Delta_k is taken as prod_i P_k, its constant factor nd^d / prod a
//     (times prod a^2 for the product peak) folded into the launch's scale fscale;
//   - for the families closed by exp (Gaussian, C0, discontinuous) the Jacobian joins the exponent:
//     |P_k| = 2^E_k m_k, so prod |P_k| = 2^(sum E_k) exp(sum ln m_k); E_k is read from the bits of
//     P_k and summed as an integer, ln m_k (tabulated per bin: below ln 2, and above -37 for a
//     subnormal P_k) is summed exactly in 64-bit fixed point, and the product costs no FP64
//     operation (the sign of prod a goes to fscale);
//   - exp and cos are table-driven (2^(j/256), cos and sin of 2 pi j / 256, filled per block), with
//     their reduced arguments' Taylor series to 2^-54 (no library constants or steps); the integer
//     k of the reduction is found in FP32 (within one of the nearest), off the FP64 pipe;
//   - the discontinuous family's cut x_i < u_i is decided exactly as defined, by one integer
//     comparison of the offset's bits with a per-bin threshold the block finds by bisection.
// The bit-level steps (c + u and yn, the bin split, exp and cos) are in fp64_bits.cuh, which also
// compiles for the host. The per-cube statistics and the reduction are the FP64 kernel's own
// (vsample.cuh: finish_block). Bin contributions (both kernels below): each sample's first (d + 1) / 2
// axes go straight to the global C with native FP64 reductions, the rest to the block's shared FP64
// copies (four lane-interleaved ones in the single-job kernel, one in the batched kernel), flushed
// into C.
#pragma once

#include <cmath>

#include "fp64_bits.cuh"
#include "vsample.cuh"

namespace mcubes {

// ln m_k of a zero-width bin (P_k = 0): the weight's factor e^-64 2^-1023 underflows with the rest
constexpr double kLogZero = -64.0;

// Families the fast FP64 kernel serves, and which per-sample closing function each takes.
template <int FID>
struct Fast64 {
    static constexpr bool kOn = FID >= 0 && FID <= 5;
    static constexpr bool kExp = FID == kGaussian || FID == kC0 || FID == kDiscontinuous;
    static constexpr bool kCos = FID == kOscillatory;
    static constexpr bool kCut = FID == kDiscontinuous;
    // the Jacobian joins the exponent (exp families): ln m_k per bin, in its own table (centred
    // families) or added to the fixed-point Q_k (the discontinuous family)
    static constexpr bool kJLog = kExp;
    // Q_k = a (B_k - u) - P_k for these, a B_k - P_k otherwise
    static constexpr bool kCentred = FID == kGaussian || FID == kC0 || FID == kProductPeak;
    // Q_k as a 64-bit fixed-point integer (2^fix_shift units), summed with integer additions
    static constexpr bool kFixedQ = !kCentred;
    static constexpr bool kLTab = kJLog && kCentred;
};

// Host: the fast kernel's per-launch parameters for family fid (0..5) at dimension d, from the
// plain FP64 parameters in Q. It serves the family when the strata fit its integer c + u (g <= 2^11)
// and the per-axis fold factors are usable: every a_i finite and non-zero (positive for C0, whose
// |a (x - u)| must equal a |x - u|) and the folded scale finite and non-zero. Q then carries the fold
// factors in ip.b (a, or a / (2 pi) for the oscillatory family), the scale nd^d / prod(fold)
// (nd^d prod a for the product peak; nd^d / prod |a| for the exp families, whose Jacobian is taken
// as prod |P_k|) and the fraction bits of the fixed-point table sums (sum_i (|fold_i| + 64) 2^fix_shift
// below 2^61 for the discontinuous family, whose sums also carry ln m_k >= kLogZero; sum_i |fold_i|
// 2^fix_shift otherwise). Returns false, leaving Q's fold fields unspecified, otherwise.
inline bool fast64_fold(int fid, VsampleParams &Q, int d)
{
    if (fid < 0 || fid > 5 || Q.g > 2048u) return false;
    constexpr double kTwoPi = 6.283185307179586;
    const bool jlog = fid == kGaussian || fid == kC0 || fid == kDiscontinuous;
    double scale = 1.0, fsum = 0.0;
    for (int i = 0; i < d; ++i) {
        const double a = Q.ip.a[i];
        if (!std::isfinite(a) || a == 0.0 || (fid == kC0 && a < 0.0)) return false;
        const double f = fid == kOscillatory ? a / kTwoPi : a;
        if (!std::isfinite(f) || f == 0.0) return false;
        Q.ip.b[i] = f;
        fsum += std::fabs(f) + (fid == kDiscontinuous ? -kLogZero : 0.0);
        scale *= (double)kNB;
        scale = fid == kProductPeak ? scale * f : scale / (jlog ? std::fabs(f) : f);
    }
    if (!std::isfinite(scale) || scale == 0.0 || !(fsum < 1e15)) return false;
    Q.fscale = scale;
    int e = 0;
    std::frexp(fsum * 1.0000001 + 1.0, &e);   // fsum + 1 < 2^e
    Q.fix_shift = 61 - e;
    return true;
}

// Block size of the single-job fast kernel: one 512-thread block an SM (16 warps, as two blocks of 256)
// holds one copy of the tables, which leaves the SM more of its L1 (frozen launches of the exp families
// ran 7-10% faster than with two 256-thread blocks). Above d = 12 the 128 registers of a 512-thread
// block would spill: 256 threads there.
__host__ __device__ constexpr int fast64_threads(int d) { return d <= 12 ? 512 : 256; }

// Axes whose bin contributions go straight to the global C (the rest use the block's shared copies).
__host__ __device__ constexpr int fast64_l2_axes(int d) { return (d + 1) / 2; }

// Shared-memory bytes of one fast FP64 block's tables: the (P, Q) table, the ln m_k table (centred
// exp families), the cut thresholds, and the exp or cos table.
template <int D, int FID>
__host__ __device__ constexpr size_t fast64_table_bytes()
{
    return (size_t)D * kNB * (16 + (Fast64<FID>::kLTab ? 8 : 0) + (Fast64<FID>::kCut ? 8 : 0)) +
           (Fast64<FID>::kExp ? kExpTab * 8 : 0) + (Fast64<FID>::kCos ? kCosTab * 16 : 0);
}

// Bytes of R copies of the FP64 bin contributions of the axes the L2 does not take.
__host__ __device__ constexpr size_t fast64_hist_bytes(int d, int r)
{
    return (size_t)r * (size_t)(d - fast64_l2_axes(d)) * kNB * 8;
}

// Copies of the shared FP64 bins in the single-job kernel, lane-interleaved: lane l adds into copy
// l mod R (word R e + l mod R of bin e), so only the lanes that share a copy can collide in one
// compare-and-swap round. A warp repeats the round while any of its lanes collided: with one copy and
// 500 random bins, 63% of warp-level updates; 20% with four. The most copies, up to 4, that keep the
// block within kFast64HistSmemCap bytes, so that the SM keeps a large L1 beside it.
constexpr size_t kFast64HistSmemCap = 164 * 1024;
template <int D, int FID>
__host__ __device__ constexpr int fast64_hist_copies()
{
    int r = 4;
    while (r > 1 && fast64_table_bytes<D, FID>() + fast64_hist_bytes(D, r) > kFast64HistSmemCap) r /= 2;
    return r;
}

// Shared-memory bytes of one single-job fast FP64 block (HK = 1: with the copies of the bins).
template <int D, int FID, int HK>
__host__ __device__ constexpr size_t fast64_smem_bytes()
{
    return fast64_table_bytes<D, FID>() + (HK == 1 ? fast64_hist_bytes(D, fast64_hist_copies<D, FID>()) : 0);
}

// Shared-memory bytes of one batched fast FP64 block (one copy of the bins).
template <int D, int FID>
__host__ __device__ constexpr size_t fast64_batch_smem_bytes()
{
    return fast64_table_bytes<D, FID>() + fast64_hist_bytes(D, 1);
}

// fast64_batch_smem_bytes (hk = 1) or the tables alone (hk = 0) at a run-time d and family (0..5), for
// host-side eligibility checks of batched classes; 0 for other families.
inline size_t fast64_smem_bytes_rt(int d, int fid, int hk)
{
    const bool cut = fid == kDiscontinuous, ex = fid == kGaussian || fid == kC0 || fid == kDiscontinuous,
               co = fid == kOscillatory, ltab = fid == kGaussian || fid == kC0;
    if (fid < 0 || fid > 5) return 0;
    return (size_t)d * kNB * (16 + (ltab ? 8 : 0) + (cut ? 8 : 0)) +
           (hk == 1 ? (size_t)(d - fast64_l2_axes(d)) * kNB * 8 : 0) + (ex ? kExpTab * 8 : 0) +
           (co ? kCosTab * 16 : 0);
}

// Stage the fast kernel's tables: per axis and bin (P, Q) (see the header), ln m_k (the exp
// families: in ltab for the centred ones, added to the fixed-point Q_k for the discontinuous one), the
// discontinuous family's cut thresholds, and the exp or cos table; clear n_hist words of the
// histogram copy. Block-wide.
template <int D, int FID>
__device__ __forceinline__ void stage_fast64(const VsampleParams &P, double2 *tab, long long *ltab, double *hist,
                                             int n_hist, unsigned long long *thr, double *ftab)
{
    const IntegrandParams &ip = P.ip;
    for (int e = threadIdx.x; e < D * kNB; e += blockDim.x) {
        const int i = e / kNB;
        const int k = e - i * kNB;
        const double b0 = P.grid[i * (kNB + 1) + k];
        const double b1 = P.grid[i * (kNB + 1) + k + 1];
        const double w = b1 - b0;
        const double a = ip.b[i];   // the fold factor (a, or a / (2 pi) for the oscillatory family)
        const double pk = a * w;
        const double base = Fast64<FID>::kCentred ? a * (b0 - ip.u[i]) : a * b0;
        // ln m_k, where |P_k| = 2^E_k m_k and E_k = (exponent field of P_k) - 1023: m_k in [1, 2), or in
        // (0, 2) for a subnormal P_k (ln m_k >= -37); kLogZero for a zero-width bin
        double lm = 0.0;
        if constexpr (Fast64<FID>::kJLog) {
            const double ap = fabs(pk);
            const int E = ((__double2hiint(ap) >> 20) & 0x7FF) - 1023;
            lm = ap > 0.0 ? log(ldexp(ap, -E)) : kLogZero;
        }
        if constexpr (Fast64<FID>::kFixedQ) {
            // |base - pk| <= |a| and |ln m_k| <= 64; the launch's fix_shift keeps the sum over the axes
            // of these bounds, times 2^fix_shift, below 2^61
            long long qf = __double2ll_rn(ldexp(base - pk, P.fix_shift));
            if constexpr (Fast64<FID>::kJLog) qf += __double2ll_rn(ldexp(lm, P.fix_shift));
            tab[e] = make_double2(pk, __longlong_as_double(qf));
        } else {
            tab[e] = make_double2(pk, base - pk);
        }
        if constexpr (Fast64<FID>::kLTab) ltab[e] = __double2ll_rn(ldexp(lm, 52));   // 2^-52 units
        if constexpr (Fast64<FID>::kCut) {
            // inside iff fma(w, delta, b0) < u; the decision is monotone in the offset, so it is a
            // threshold on the offset's bit pattern: yn's bits in bin 0, G's bits in the others,
            // where the offset is a multiple of 2^(e - 52), e the exponent of yn in bin k.
            const double u = ip.u[i];
            unsigned long long t;
            if (k == 0) {
                // smallest yn in [0, 1) with fma(w, yn, 0) >= u (2^62 bit patterns: bisection)
                unsigned long long lo = 0ull, hi = 0x3FF0000000000000ull;   // bits(1.0): outside the bin
                while (lo < hi) {
                    const unsigned long long mid = lo + ((hi - lo) >> 1);
                    if (__fma_rn(w, __longlong_as_double((long long)mid), b0) >= u) hi = mid;
                    else lo = mid + 1;
                }
                t = lo;
            } else {
                const int ex = 31 - __clz(k);                  // exponent of yn in [k, k + 1)
                const int sh = 52 - ex;                        // fraction bits of the offset
                const double step = __longlong_as_double((long long)(1023 - sh) << 52);   // 2^-sh
                unsigned long long lo = 0ull, hi = 1ull << sh;  // offset j step, j in [0, 2^sh)
                while (lo < hi) {
                    const unsigned long long mid = lo + ((hi - lo) >> 1);
                    if (__fma_rn(w, (double)mid * step, b0) >= u) hi = mid;
                    else lo = mid + 1;
                }
                // G = 1 + j step has fraction bits j << (52 - sh)
                t = lo >= (1ull << sh) ? 0x4000000000000000ull : (0x3FF0000000000000ull | (lo << (52 - sh)));
            }
            thr[e] = t;   // inside iff bits < t
        }
    }
    if constexpr (Fast64<FID>::kExp) {
        for (int j = threadIdx.x; j < kExpTab; j += blockDim.x) ftab[j] = exp2((double)j / (double)kExpTab);
    }
    if constexpr (Fast64<FID>::kCos) {
        double2 *cs = reinterpret_cast<double2 *>(ftab);
        for (int j = threadIdx.x; j < kCosTab; j += blockDim.x) {
            double s, c;
            sincospi((double)j / (double)(kCosTab / 2), &s, &c);
            cs[j] = make_double2(c, s);
        }
    }
    for (int e = threadIdx.x; e < n_hist; e += blockDim.x) hist[e] = 0.0;
    __syncthreads();
}

// Algorithm 2's loop over sub-cubes [t, t_end) for the fast FP64 kernel.
template <int D, int FID, int HK, int kR>
__device__ __forceinline__ void sample_cubes_fast64(const VsampleParams &P, const PhiloxPre &ph, uint32_t t,
                                                    const uint32_t t_end,
                                                    const double2 *tab, const long long *ltab, double *hist,
                                                    const unsigned long long *thr, const double *ftab,
                                                    ThreadSums &acc)
{
    static_assert(Fast64<FID>::kOn, "the fast FP64 kernel serves the six Genz families");
    static_assert(kR >= 1 && (kR & (kR - 1)) == 0, "a power of two of copies");
    const bool adjust = HK == 1 && P.adjust != 0;
    const int copy = (int)(threadIdx.x & (unsigned)(kR - 1));   // this lane's copy of the shared bins
    // strata digits c_i, held as c_i 2^20 (the high word of c_i 2^52; g <= 2^11)
    uint32_t dsh[D];
    {
        uint32_t rest = t;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            dsh[i] = (rest % P.g) << 20;
            rest /= P.g;
        }
    }
    const uint32_t gsh = P.g << 20;
    const double inv_fix = ldexp(1.0, -P.fix_shift);
    const unsigned long long Rb = (unsigned long long)__double_as_longlong(P.R);
    const unsigned long long Rm = (Rb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int eR = (int)(Rb >> 52) - 1023;   // R = nd / g >= 500 / 2048: normal
    const unsigned long long ycap_bits = (unsigned long long)__double_as_longlong(P.ycap);
    const uint32_t p = P.p;
    const double s0 = FID == kOscillatory ? P.ip.u[0] : 0.0;   // the phase offset u_1, in turns
    constexpr int kCalls = (D + 1) / 2;

    for (; t < t_end; ++t) {
        if (!mc_check(P.chk, t, P.m, 3)) break;
        double S1 = 0.0, S2 = 0.0;
        const PhiloxCube cube = philox_cube(t, ph);
        for (uint32_t q = 0; q < p; ++q) {
            double s = s0, prod = 1.0, J = 1.0;
            long long sq = 0;   // fixed-point sum of the Q_k (kFixedQ; with the ln m_k for kJLog)
            long long sl = 0;   // sum of the ln m_k, 2^-52 units (kLTab)
            int sE = 0;         // sum of the exponent fields of the P_k (kJLog)
            bool inside = true;
            int kofs[D];
#pragma unroll
            for (int j = 0; j < kCalls; ++j) {
                const Words4 r = philox_draw(q, j, cube, ph);
                const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = 2 * j + h;
                    if (i < D) {
                        unsigned long long yb = cu_times_r_bits(dsh[i] | (wv[2 * h] & 0xFFFFFu), wv[2 * h + 1], Rm, eR);
                        yb = yb < ycap_bits ? yb : ycap_bits;   // min(yn, largest double below nd)
                        unsigned long long gb;
                        int k = split_bin(yb, gb);
                        if (!mc_check(P.chk, k, kNB, 1)) k = 0;
                        kofs[i] = i * kNB + k;
                        const double2 pq = tab[kofs[i]];
                        const double G = __longlong_as_double((long long)gb);
                        if constexpr (Fast64<FID>::kJLog) sE += (__double2hiint(pq.x) >> 20) & 0x7FF;
                        if constexpr (Fast64<FID>::kLTab) sl += ltab[kofs[i]];
                        if constexpr (Fast64<FID>::kFixedQ) {
                            s = __fma_rn(pq.x, G, s);
                            sq += __double_as_longlong(pq.y);
                        } else {
                            const double v = __fma_rn(pq.x, G, pq.y);
                            if constexpr (FID == kGaussian) {
                                s = __fma_rn(v, v, s);
                            } else if constexpr (FID == kC0) {
                                s += fabs(v);
                            } else {   // product peak
                                prod *= __fma_rn(v, v, 1.0);
                            }
                        }
                        if constexpr (Fast64<FID>::kCut) inside = inside && ((k == 0 ? yb : gb) < thr[kofs[i]]);
                        if constexpr (!Fast64<FID>::kJLog) J *= pq.x;
                    }
                }
            }
            if constexpr (Fast64<FID>::kFixedQ) s = __fma_rn(__ll2double_rn(sq), inv_fix, s);
            // the exp families' weight f prod |P_k| = 2^(sum E_k) exp(+-s + sum ln m_k)
            const int E = sE - D * 1023;
            double fv;
            if constexpr (FID == kGaussian || FID == kC0) {
                fv = exp_tab(__fma_rn(__ll2double_rn(sl), 0x1p-52, -s), E, ftab);
            } else if constexpr (FID == kDiscontinuous) {
                fv = inside ? exp_tab(s, E, ftab) : 0.0;
            } else if constexpr (FID == kOscillatory) {
                fv = cos_turns(s, reinterpret_cast<const double2 *>(ftab));
            } else if constexpr (FID == kProductPeak) {
                fv = __drcp_rn(prod);
            } else {   // corner peak
                fv = inv_pow<D + 1>(1.0 + s);
            }
            const double w = Fast64<FID>::kJLog ? fv : fv * J;   // the weight without the launch's scale fscale
            S1 += w;
            S2 = __fma_rn(w, w, S2);
            if (adjust) {
                const double wf = w * P.fscale;
                const double hv = wf * wf;
                // The first kL2 axes: native FP64 reductions into the global C, which the L2 performs, off
                // the FP64 pipe. The rest: this lane's copy of the block's shared bins, whose atomics are
                // compare-and-swap loops around an FP64 add on the SM. Half and half keeps the launch time the
                // same wherever C lies (the L2's reduction rate into C depends on its physical placement). A
                // zero adds nothing.
                if (hv != 0.0) {
                    constexpr int kL2 = fast64_l2_axes(D);
#pragma unroll
                    for (int i = 0; i < kL2; ++i) red_add_f64_global(&P.C[kofs[i]], hv);
#pragma unroll
                    for (int i = kL2; i < D; ++i) atomicAdd(&hist[(kofs[i] - kL2 * kNB) * kR + copy], hv);
                }
            }
        }
        const bool probe_this = P.probe != nullptr && (t & P.probe_mask) == 0 &&
                                mc_check(P.chk, t >> P.probe_shift, (long long)(P.m >> P.probe_shift) + 1, 4);
        const double It = S1 * P.inv_p;
        double Vt = __fma_rn(-It, S1, S2);
        Vt = Vt > 0.0 ? Vt : 0.0;
        acc.sI += It;
        acc.sV += Vt;
        if (probe_this) {
            P.probe[2 * (size_t)(t >> P.probe_shift)] = It * P.fscale;
            P.probe[2 * (size_t)(t >> P.probe_shift) + 1] = Vt * P.inv_pp1 * P.fscale * P.fscale;
        }
        bool carry = true;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if (carry) {
                dsh[i] += 1u << 20;
                if (dsh[i] < gsh) {
                    carry = false;
                } else {
                    dsh[i] = 0u;
                }
            }
        }
    }
}

// Add the block's kR lane-interleaved copies of the shared bins (axes fast64_l2_axes(D)..D-1) into C,
// the copies of a bin summed in order; block-wide, ends with a barrier so that the copies can be
// cleared again.
template <int D, int kR>
__device__ __forceinline__ void flush_fast64_hist(double *C, const double *hist)
{
    constexpr int kL2 = fast64_l2_axes(D);
    for (int e = threadIdx.x; e < (D - kL2) * kNB; e += blockDim.x) {
        double v = hist[(size_t)e * kR];
#pragma unroll
        for (int c = 1; c < kR; ++c) v += hist[(size_t)e * kR + c];
        if (v != 0.0) atomicAdd(&C[kL2 * kNB + e], v);
    }
    __syncthreads();
}

// One job, persistent grid; HK = 0 frozen, HK = 1 adjusting. Adjusting launches add each sample's
// contribution on half its axes straight into the job's FP64 C with native FP64 reductions, which the
// L2 performs (off the FP64 pipe, the kernel's bound), and on the other half into the block's
// lane-interleaved shared FP64 copies (fast64_hist_copies), flushed into C at the end.
template <int D, int FID, int HK>
__global__ void __launch_bounds__(fast64_threads(D), 1) vsample_fast64_kernel(const VsampleParams P)
{
    constexpr int kL2 = fast64_l2_axes(D);
    constexpr int kR = fast64_hist_copies<D, FID>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *tab = reinterpret_cast<double2 *>(smem_raw);
    unsigned char *next = smem_raw + (size_t)D * kNB * 16;
    long long *ltab = reinterpret_cast<long long *>(next);
    if constexpr (Fast64<FID>::kLTab) next += (size_t)D * kNB * 8;
    double *hist = reinterpret_cast<double *>(next);
    if constexpr (HK == 1) next += fast64_hist_bytes(D, kR);
    unsigned long long *thr = reinterpret_cast<unsigned long long *>(next);
    if constexpr (Fast64<FID>::kCut) next += (size_t)D * kNB * 8;
    double *ftab = reinterpret_cast<double *>(next);
    __shared__ double red_scratch[64];

    const bool adjust = HK == 1 && P.adjust != 0;
    stage_fast64<D, FID>(P, tab, ltab, hist, adjust ? (D - kL2) * kNB * kR : 0, thr, ftab);

    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t rng = (gtid * (uint64_t)P.perm_mul) % nthreads;
    const uint32_t t = (uint32_t)((rng * P.m) / nthreads);
    const uint32_t t_end = (uint32_t)(((rng + 1) * P.m) / nthreads);

    ThreadSums acc;
    sample_cubes_fast64<D, FID, HK, kR>(P, P.ph, t, t_end, tab, ltab, hist, thr, ftab, acc);
    const IntHist none{0u, 0u, 0u, 0.0f, 0.0f};
    finish_block<D, false, HK>(P, acc, hist, none, false, 1.0f, red_scratch);
    if (adjust) flush_fast64_hist<D, kR>(P.C, hist);
}

// ------------------------------------------------------------------------------ batches
// The batched form (the batch kernel's tiling: block b takes the contiguous tile range
// [b n / B, (b+1) n / B) of one (d, family) class and switches job only at job boundaries) for
// classes whose jobs all take the fast kernel. On each switch the block flushes the finished job's
// sums and shared copy, stages the next job's folded tables and prepares its Philox launch constants
// (for this iteration) in shared memory. Adjusting iterations route the bin contributions as the
// single-job kernel does: half the axes to each job's global C with native FP64 reductions, half to
// the shared copy. Each job's parameters carry its fold (fast64_fold on the host).
template <int D, int FID>
__global__ void __launch_bounds__(kMaxBlockThreads, 1)
    vsample_batch_fast64_kernel(const BatchJob *__restrict__ jobs, const BatchTile *__restrict__ tiles, int n_tiles,
                                int iteration, int parity, int adjust, uint32_t perm_mul)
{
    constexpr int kL2 = fast64_l2_axes(D);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *tab = reinterpret_cast<double2 *>(smem_raw);
    unsigned char *next = smem_raw + (size_t)D * kNB * 16;
    long long *ltab = reinterpret_cast<long long *>(next);
    if constexpr (Fast64<FID>::kLTab) next += (size_t)D * kNB * 8;
    double *hist = reinterpret_cast<double *>(next);
    next += (size_t)(D - kL2) * kNB * 8;
    unsigned long long *thr = reinterpret_cast<unsigned long long *>(next);
    if constexpr (Fast64<FID>::kCut) next += (size_t)D * kNB * 8;
    double *ftab = reinterpret_cast<double *>(next);
    __shared__ double red_scratch[64];
    __shared__ PhiloxPre ph;

    const int tb = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
    const int te = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
    const uint32_t r = (uint32_t)(((uint64_t)threadIdx.x * perm_mul) % blockDim.x);
    const IntHist none{0u, 0u, 0u, 0.0f, 0.0f};

    int cur = -1;
    VsampleParams P;
    ThreadSums acc;
    for (int ti = tb; ti < te; ++ti) {
        const BatchTile tile = tiles[ti];
        if ((int)tile.job != cur) {
            if (cur >= 0) {
                finish_block<D, false, 1>(P, acc, hist, none, false, 1.0f, red_scratch);
                if (adjust) flush_fast64_hist<D, 1>(P.C, hist);
                acc = ThreadSums();
            }
            cur = (int)tile.job;
            const BatchJob &J = jobs[cur];
            P = J.P;
            P.grid = J.grid[parity];
            P.C = J.C;
            P.sums = J.sums + 2 * iteration;
            P.prev = nullptr;
            P.ctr2_hi = (uint32_t)iteration << 16;
            P.adjust = adjust;
            P.probe = nullptr;
            if (threadIdx.x == 0) philox_prepare(ph, P.key0, P.key1, P.ctr2_hi, P.job);
            stage_fast64<D, FID>(P, tab, ltab, hist, adjust ? (D - kL2) * kNB : 0, thr, ftab);   // ends with a barrier
        }
        if (!mc_check(P.chk, (long long)tile.c1 - 1, P.m, 5) || !mc_check(P.chk, tile.c0, (long long)tile.c1, 5)) continue;
        const uint32_t n = tile.c1 - tile.c0;
        const uint32_t t = tile.c0 + (uint32_t)(((uint64_t)r * n) / blockDim.x);
        const uint32_t t_end = tile.c0 + (uint32_t)(((uint64_t)(r + 1) * n) / blockDim.x);
        sample_cubes_fast64<D, FID, 1, 1>(P, ph, t, t_end, tab, ltab, hist, thr, ftab, acc);
    }
    if (cur >= 0) {
        finish_block<D, false, 1>(P, acc, hist, none, false, 1.0f, red_scratch);
        if (adjust) flush_fast64_hist<D, 1>(P.C, hist);
    }
}

}  // namespace mcubes
