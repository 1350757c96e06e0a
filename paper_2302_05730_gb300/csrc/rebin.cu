// Grid refinement ("Rebin") of the VEGAS importance grid that m-Cubes adapts (paper Sec. 3.2,
// which delegates the rule to VEGAS, Lepage 1978). One block of 512 threads per axis (and, in
// the batched form, per job and axis), FP64:
//   1. smooth the bin contributions with a 3-point average (2-point at the ends);
//   2. normalise by their sum D (an axis with D = 0 or non-finite keeps its grid);
//   3. damp: r_k = ((1 - rho_k) / ln(1/rho_k))^alpha, rho_k = d_k / D (r = 0 for an empty
//      bin, 1 when one bin holds everything);
//   4. running sums R_k of r (one warp, 16 bins per lane, then a shuffle scan);
//   5. place new boundary l at damped mass l S / nd: find the bin k with R_k <= l S/nd <
//      R_{k+1} by binary search, and interpolate linearly inside it (fraction cut to [0, 1]).
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace mcubes {

constexpr int kRebinThreads = 512;

// One axis: Bi (501 boundaries), Ci (500 contributions) -> Bo. Block-wide, 512 threads.
__device__ __forceinline__ void rebin_axis(const double *__restrict__ Bi, const double *__restrict__ Ci,
                                           double *__restrict__ Bo, double alpha)
{
    __shared__ double Bs[kNB + 1];
    __shared__ double Cs[kNB];
    __shared__ double rs[kNB];
    __shared__ double Rs[kNB + 1];
    __shared__ double wsum[kRebinThreads / 32];
    __shared__ int keep;

    const int tid = threadIdx.x;

    for (int k = tid; k <= kNB; k += blockDim.x) Bs[k] = Bi[k];
    for (int k = tid; k < kNB; k += blockDim.x) Cs[k] = Ci[k];
    __syncthreads();

    // 1. smoothing
    double dk = 0.0;
    if (tid < kNB) {
        if (tid == 0) dk = (Cs[0] + Cs[1]) / 2.0;
        else if (tid == kNB - 1) dk = (Cs[kNB - 2] + Cs[kNB - 1]) / 2.0;
        else dk = (Cs[tid - 1] + Cs[tid] + Cs[tid + 1]) / 3.0;
    }

    // 2. D = sum of smoothed contributions (fixed-order tree)
    double v = dk;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) wsum[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double D = 0.0;
        for (int w = 0; w < kRebinThreads / 32; ++w) D += wsum[w];
        wsum[0] = D;
        keep = !(D > 0.0) || !isfinite(D);
    }
    __syncthreads();
    const double D = wsum[0];
    if (keep) {
        for (int k = tid; k <= kNB; k += blockDim.x) Bo[k] = Bs[k];
        return;
    }

    // 3. damping
    if (tid < kNB) {
        const double rho = dk / D;
        double r;
        if (dk == 0.0) r = 0.0;
        else if (rho == 1.0) r = 1.0;
        else r = pow((1.0 - rho) / (-log(rho)), alpha);
        rs[tid] = r;
    }
    __syncthreads();

    // 4. running sums R_0 = 0, R_{k+1} = R_k + r_k: lane L of warp 0 owns bins [16 L, 16 L + 16)
    if (tid < 32) {
        constexpr int kPer = (kNB + 31) / 32;   // 16
        const int k0 = tid * kPer;
        double part = 0.0;
        for (int k = k0; k < k0 + kPer && k < kNB; ++k) part += rs[k];
        double incl = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double n = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += n;
        }
        double run = incl - part;   // exclusive prefix of this lane
        for (int k = k0; k < k0 + kPer && k < kNB; ++k) {
            Rs[k] = run;
            run += rs[k];
        }
        if (tid == 31) Rs[kNB] = run;
    }
    __syncthreads();

    // 5. new boundaries at equal damped mass
    const double S = Rs[kNB];
    for (int l = tid; l <= kNB; l += blockDim.x) {
        double b;
        if (l == 0) {
            b = 0.0;
        } else if (l == kNB) {
            b = 1.0;
        } else {
            const double T = (double)l * S / (double)kNB;
            // largest k in [0, nd-1] with R_k <= T
            int lo = 0, hi = kNB - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (Rs[mid] <= T) lo = mid; else hi = mid - 1;
            }
            const int k = lo;
            const double rk = rs[k];
            double frac = rk > 0.0 ? (T - Rs[k]) / rk : 0.0;
            frac = frac > 1.0 ? 1.0 : (frac < 0.0 ? 0.0 : frac);
            b = Bs[k] + (Bs[k + 1] - Bs[k]) * frac;
        }
        Bo[l] = b;
    }
}

__global__ void __launch_bounds__(kRebinThreads) rebin_kernel(const double *__restrict__ grid_in,
                                                            const double *__restrict__ C,
                                                            double *__restrict__ grid_out,
                                                            double alpha)
{
    const int axis = blockIdx.x;
    rebin_axis(grid_in + (size_t)axis * (kNB + 1), C + (size_t)axis * kNB, grid_out + (size_t)axis * (kNB + 1),
               alpha);
}

// Many (job, axis) pairs: block b refines axis block_axis[b] of job block_job[b].
__global__ void __launch_bounds__(kRebinThreads) rebin_batch_kernel(const uint32_t *__restrict__ block_job,
                                                                  const uint32_t *__restrict__ block_axis,
                                                                  const double *const *__restrict__ grid_in,
                                                                  const double *const *__restrict__ C,
                                                                  double *const *__restrict__ grid_out,
                                                                  double alpha)
{
    const uint32_t j = block_job[blockIdx.x];
    const uint32_t a = block_axis[blockIdx.x];
    rebin_axis(grid_in[j] + (size_t)a * (kNB + 1), C[j] + (size_t)a * kNB, grid_out[j] + (size_t)a * (kNB + 1),
               alpha);
}

int launch_rebin(int d, const double *d_grid_in, const double *d_C, double *d_grid_out,
                 double alpha, cudaStream_t stream)
{
    rebin_kernel<<<d, kRebinThreads, 0, stream>>>(d_grid_in, d_C, d_grid_out, alpha);
    return (int)cudaGetLastError();
}

int launch_rebin_batch(int n_blocks, const uint32_t *block_job, const uint32_t *block_axis,
                       const double *const *grid_in, const double *const *C, double *const *grid_out,
                       double alpha, cudaStream_t stream)
{
    if (n_blocks <= 0) return (int)cudaSuccess;
    rebin_batch_kernel<<<n_blocks, kRebinThreads, 0, stream>>>(block_job, block_axis, grid_in, C, grid_out, alpha);
    return (int)cudaGetLastError();
}

}  // namespace mcubes
