// Learned proposal for m-Cubes: a coupling flow on [0,1]^d with piecewise-quadratic CDFs whose
// parameters come from a small ReLU MLP per layer (neural importance sampling). It stands in
// for the separable VEGAS grid on correlated integrands.
//
// Parameter layout, per layer l (FP32 master copy, flat): W1 [H x |A|], b1 [H], W2 [H x H], b2 [H],
// W3 [Nout x H], b3 [Nout] with Nout = |B| (2K + 1). Output slot s (axis B[s]) holds K
// unnormalised bin widths, then K+1 unnormalised edge values.
// Axis split of layer l: l mod 4 = 0 -> A = first floor(d/2) axes; 1 -> swapped; 2 -> A = even
// axes; 3 -> swapped.
//
// MLP: BF16 operands, FP32 accumulation, on the tensor cores through mma.sync m16n8k16. A CTA
// takes 64 samples (4 warps x 16 rows); weights and activations are staged in shared memory
// k-contiguous, with rows padded by 8 elements so fragment loads are conflict-free.
// Coupling transform: FP32 SIMT, one thread per sample.
//
// The kernels of one layer exchange activations through global memory (o, r1, r2, dz1, dz2,
// dL/do). The gradient of a training step is the exact gradient of the flow's loss, up to
// the bf16 rounding of the MLP operands.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/mcubes.h"
#include "flow_common.cuh"
#include "internal.h"

namespace mcubes {
namespace flow {

// ------------------------------------------------------------------------------ mma helpers
// acc[nt] (16 x 8 blocks) += A[16 x K] * B[K x 8 NT] for this warp, where A is row-major
// (k contiguous, row stride lda) and B is given transposed, BT[n][k] (row stride ldb).
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4):
//   A regs: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
//   B regs: (k 2t..2t+1, n g), (k 2t+8.., n g)
//   C: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
template <int NT>
__device__ __forceinline__ void warp_mma(float (&acc)[NT][4], const __nv_bfloat16 *A, int lda,
                                         const __nv_bfloat16 *BT, int ldb, int K)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        a[0] = ld32(A + g * lda + k0 + 2 * t);
        a[1] = ld32(A + (g + 8) * lda + k0 + 2 * t);
        a[2] = ld32(A + g * lda + k0 + 8 + 2 * t);
        a[3] = ld32(A + (g + 8) * lda + k0 + 8 + 2 * t);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const __nv_bfloat16 *bp = BT + (nt * 8 + g) * ldb + k0 + 2 * t;
            mma16816(acc[nt], a, ld32(bp), ld32(bp + 8));
        }
    }
}

// Stage a [rows x cols] FP32 matrix (row-major, global) as bf16 into dst[r * ld + c], zero-padding
// rows up to rows_p and cols up to cols_p. transpose: dst[c * ld + r] instead.
__device__ __forceinline__ void stage_bf16(__nv_bfloat16 *dst, int ld, const float *src, int rows, int cols,
                                           int rows_p, int cols_p, bool transpose)
{
    for (int e = threadIdx.x; e < rows_p * cols_p; e += blockDim.x) {
        const int r = e / cols_p, c = e - r * cols_p;
        const float v = (r < rows && c < cols) ? src[(size_t)r * cols + c] : 0.0f;
        if (transpose) dst[c * ld + r] = __float2bfloat16_rn(v);
        else dst[r * ld + c] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------------------------ MLP forward
// o = W3 relu(W2 relu(W1 a + b1) + b2) + b3 for the samples of this tile, a = h[s][A].
// Writes o (n x nout FP32); when r1/r2 are given, also the bf16 activations (n x H).
template <int H>
__global__ void __launch_bounds__(128) mlp_fwd_kernel(const float *__restrict__ params, const LayerDesc D,
                                                      const float *__restrict__ h, int d, long long n,
                                                      float *__restrict__ o, __nv_bfloat16 *__restrict__ r1g,
                                                      __nv_bfloat16 *__restrict__ r2g)
{
    constexpr int LD0 = kK0 + 8, LDH = H + 8;
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *W1 = reinterpret_cast<__nv_bfloat16 *>(sm);        // [H][LD0]
    __nv_bfloat16 *W2 = W1 + H * LD0;                                   // [H][LDH]
    __nv_bfloat16 *W3 = W2 + H * LDH;                                   // [nout_p][LDH]
    __nv_bfloat16 *a0 = W3 + D.nout_p * LDH;                            // [64][LD0]
    __nv_bfloat16 *r1 = a0 + kTileRows * LD0;                           // [64][LDH]
    __nv_bfloat16 *r2 = r1 + kTileRows * LDH;                           // [64][LDH]
    float *b1 = reinterpret_cast<float *>(r2 + kTileRows * LDH);
    float *b2 = b1 + H;
    float *b3 = b2 + H;                                                 // [nout_p]

    stage_bf16(W1, LD0, params + D.offW1, H, D.nA, H, kK0, false);
    stage_bf16(W2, LDH, params + D.offW2, H, H, H, H, false);
    stage_bf16(W3, LDH, params + D.offW3, D.nout, H, D.nout_p, H, false);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        b1[i] = params[D.offb1 + i];
        b2[i] = params[D.offb2 + i];
    }
    for (int i = threadIdx.x; i < D.nout_p; i += blockDim.x) b3[i] = i < D.nout ? params[D.offb3 + i] : 0.0f;
    const long long row0 = (long long)blockIdx.x * kTileRows;
    for (int e = threadIdx.x; e < kTileRows * kK0; e += blockDim.x) {
        const int r = e / kK0, c = e - r * kK0;
        const long long s = row0 + r;
        const float v = (s < n && c < D.nA) ? h[s * d + D.A[c]] : 0.0f;
        a0[r * LD0 + c] = __float2bfloat16_rn(v);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int wr = warp * 16;
    const long long sA = row0 + wr + g, sB = sA + 8;
    {   // layer 1
        float acc[H / 8][4] = {};
        warp_mma<H / 8>(acc, a0 + wr * LD0, LD0, W1, LD0, kK0);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            const uint32_t top = pack_bf16(fmaxf(acc[nt][0] + b1[c], 0.f), fmaxf(acc[nt][1] + b1[c + 1], 0.f));
            const uint32_t bot = pack_bf16(fmaxf(acc[nt][2] + b1[c], 0.f), fmaxf(acc[nt][3] + b1[c + 1], 0.f));
            *reinterpret_cast<uint32_t *>(r1 + (wr + g) * LDH + c) = top;
            *reinterpret_cast<uint32_t *>(r1 + (wr + g + 8) * LDH + c) = bot;
            if (r1g) {
                if (sA < n) *reinterpret_cast<uint32_t *>(r1g + sA * H + c) = top;
                if (sB < n) *reinterpret_cast<uint32_t *>(r1g + sB * H + c) = bot;
            }
        }
    }
    __syncwarp();
    {   // layer 2
        float acc[H / 8][4] = {};
        warp_mma<H / 8>(acc, r1 + wr * LDH, LDH, W2, LDH, H);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            const uint32_t top = pack_bf16(fmaxf(acc[nt][0] + b2[c], 0.f), fmaxf(acc[nt][1] + b2[c + 1], 0.f));
            const uint32_t bot = pack_bf16(fmaxf(acc[nt][2] + b2[c], 0.f), fmaxf(acc[nt][3] + b2[c + 1], 0.f));
            *reinterpret_cast<uint32_t *>(r2 + (wr + g) * LDH + c) = top;
            *reinterpret_cast<uint32_t *>(r2 + (wr + g + 8) * LDH + c) = bot;
            if (r2g) {
                if (sA < n) *reinterpret_cast<uint32_t *>(r2g + sA * H + c) = top;
                if (sB < n) *reinterpret_cast<uint32_t *>(r2g + sB * H + c) = bot;
            }
        }
    }
    __syncwarp();
    // layer 3, in chunks of 8 output tiles
    for (int n0 = 0; n0 < D.nout_p; n0 += 64) {
        float acc[8][4] = {};
        const int nts = min(8, (D.nout_p - n0) / 8);
        if (nts == 8) {
            warp_mma<8>(acc, r2 + wr * LDH, LDH, W3 + n0 * LDH, LDH, H);
        } else {
            for (int j = 0; j < nts; ++j) {
                float one[1][4] = {};
                warp_mma<1>(one, r2 + wr * LDH, LDH, W3 + (n0 + j * 8) * LDH, LDH, H);
                acc[j][0] = one[0][0]; acc[j][1] = one[0][1]; acc[j][2] = one[0][2]; acc[j][3] = one[0][3];
            }
        }
        // scalar stores: a row holds nout = |B| (2K+1) values, odd when |B| is odd, so neither
        // 8-byte alignment nor c + 1 < nout can be assumed
        for (int nt = 0; nt < nts; ++nt) {
            const int c = n0 + nt * 8 + 2 * t;
            if (sA < n) {
                if (c < D.nout) o[sA * D.nout + c] = acc[nt][0] + b3[c];
                if (c + 1 < D.nout) o[sA * D.nout + c + 1] = acc[nt][1] + b3[c + 1];
            }
            if (sB < n) {
                if (c < D.nout) o[sB * D.nout + c] = acc[nt][2] + b3[c];
                if (c + 1 < D.nout) o[sB * D.nout + c + 1] = acc[nt][3] + b3[c + 1];
            }
        }
    }
}

template <int H>
size_t mlp_fwd_smem(const LayerDesc &D)
{
    constexpr int LD0 = kK0 + 8, LDH = H + 8;
    return sizeof(__nv_bfloat16) * ((size_t)H * LD0 + (size_t)H * LDH + (size_t)D.nout_p * LDH + kTileRows * LD0 +
                                     2 * kTileRows * LDH) +
           sizeof(float) * (2 * H + D.nout_p);
}

// ------------------------------------------------------------------------------ coupling
// mode 0: density direction (y = CDF(x)); mode 1: sampling direction (x = CDF^-1(y)).
// h_in -> h_out for the B axes (A axes copied); logq += log pdf.
template <int K>
__global__ void coupling_kernel(const LayerDesc D, const float *__restrict__ o, const float *__restrict__ h_in,
                                float *__restrict__ h_out, float *__restrict__ logq, int d, long long n, int mode)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        float lq = 0.f;
        for (int a = 0; a < D.nA; ++a) h_out[s * d + D.A[a]] = h_in[s * d + D.A[a]];
        for (int j = 0; j < D.nB; ++j) {
            const float *raw = o + s * D.nout + j * (2 * K + 1);
            float out, q;
            pq_transform<K>(raw, h_in[s * d + D.B[j]], mode, out, q);
            h_out[s * d + D.B[j]] = out;
            lq += __logf(q);
        }
        logq[s] += lq;
    }
}

// Backward of one coupling layer (density direction). In: the layer input h_in, the MLP output o,
// the gradient gout = dL/dh_out (n x d) and gl = dL/dlogq (n). Out: dL/do (n x nout), and
// gin = dL/dh_in for the B axes plus the pass-through of the A axes (the MLP part of the A axes is
// added by the backward-data kernel).
template <int K>
__global__ void coupling_bwd_kernel(const LayerDesc D, const float *__restrict__ o, const float *__restrict__ h_in,
                                    const float *__restrict__ gout, const float *__restrict__ gl,
                                    float *__restrict__ dodraw, float *__restrict__ gin, int d, long long n)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const float glq = gl[s];
        for (int a = 0; a < D.nA; ++a) gin[s * d + D.A[a]] = gout[s * d + D.A[a]];
        for (int j = 0; j < D.nB; ++j) {
            const float *raw = o + s * D.nout + j * (2 * K + 1);
            float *draw = dodraw + s * D.nout + j * (2 * K + 1);
            gin[s * d + D.B[j]] = pq_backward<K>(raw, h_in[s * d + D.B[j]], gout[s * d + D.B[j]], glq,
                                                 [draw](int k, float v) { draw[k] = v; });
        }
    }
}

// ------------------------------------------------------------------------------ MLP backward
// dr2 = dL/do W3, dz2 = dr2 * (r2 > 0), dr1 = dz2 W2, dz1 = dr1 * (r1 > 0), da = dz1 W1.
// Writes dz1, dz2 (bf16, n x H) and adds da to gin[s][A].
template <int H>
__global__ void __launch_bounds__(128) mlp_bwd_data_kernel(const float *__restrict__ params, const LayerDesc D,
                                                           const float *__restrict__ dodraw,
                                                           const __nv_bfloat16 *__restrict__ r1g,
                                                           const __nv_bfloat16 *__restrict__ r2g, long long n, int d,
                                                           __nv_bfloat16 *__restrict__ dz1g,
                                                           __nv_bfloat16 *__restrict__ dz2g, float *__restrict__ gin)
{
    constexpr int LDH = H + 8;
    const int LDO = D.nout_p + 8;
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *W3T = reinterpret_cast<__nv_bfloat16 *>(sm);      // [H][LDO]: W3T[h][o] = W3[o][h]
    __nv_bfloat16 *W2T = W3T + H * LDO;                                // [H][LDH]: W2T[i][o] = W2[o][i]
    __nv_bfloat16 *W1T = W2T + H * LDH;                                // [8][LDH]: W1T[c][h] = W1[h][c]
    __nv_bfloat16 *gO = W1T + 8 * LDH;                                 // [64][LDO]
    __nv_bfloat16 *dz2 = gO + kTileRows * LDO;                         // [64][LDH]

    stage_bf16(W3T, LDO, params + D.offW3, D.nout, H, D.nout_p, H, true);
    stage_bf16(W2T, LDH, params + D.offW2, H, H, H, H, true);
    stage_bf16(W1T, LDH, params + D.offW1, H, D.nA, H, 8, true);
    const long long row0 = (long long)blockIdx.x * kTileRows;
    for (int e = threadIdx.x; e < kTileRows * D.nout_p; e += blockDim.x) {
        const int r = e / D.nout_p, c = e - r * D.nout_p;
        const long long s = row0 + r;
        const float v = (s < n && c < D.nout) ? dodraw[s * D.nout + c] : 0.0f;
        gO[r * LDO + c] = __float2bfloat16_rn(v);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int wr = warp * 16;
    const long long sA = row0 + wr + g, sB = sA + 8;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    auto relu_mask = [&](const __nv_bfloat16 *rg, long long s, int c, float v0, float v1, float &m0, float &m1) {
        if (s < n) {
            const __nv_bfloat162 r = *reinterpret_cast<const __nv_bfloat162 *>(rg + s * H + c);
            m0 = __hgt(r.x, zero) ? v0 : 0.f;
            m1 = __hgt(r.y, zero) ? v1 : 0.f;
        } else {
            m0 = m1 = 0.f;
        }
    };
    {
        float acc[H / 8][4] = {};
        warp_mma<H / 8>(acc, gO + wr * LDO, LDO, W3T, LDO, D.nout_p);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            float a0, a1, a2, a3;
            relu_mask(r2g, sA, c, acc[nt][0], acc[nt][1], a0, a1);
            relu_mask(r2g, sB, c, acc[nt][2], acc[nt][3], a2, a3);
            const uint32_t top = pack_bf16(a0, a1), bot = pack_bf16(a2, a3);
            *reinterpret_cast<uint32_t *>(dz2 + (wr + g) * LDH + c) = top;
            *reinterpret_cast<uint32_t *>(dz2 + (wr + g + 8) * LDH + c) = bot;
            if (sA < n) *reinterpret_cast<uint32_t *>(dz2g + sA * H + c) = top;
            if (sB < n) *reinterpret_cast<uint32_t *>(dz2g + sB * H + c) = bot;
        }
    }
    __syncwarp();
    // dz1 reuses this warp's own rows of gO (16 rows of stride LDO hold 16 rows of stride LDH)
    __nv_bfloat16 *dz1 = gO + wr * LDO;
    {
        float acc[H / 8][4] = {};
        warp_mma<H / 8>(acc, dz2 + wr * LDH, LDH, W2T, LDH, H);
        __syncwarp();   // all lanes done reading this warp's gO rows before overwriting them
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            float a0, a1, a2, a3;
            relu_mask(r1g, sA, c, acc[nt][0], acc[nt][1], a0, a1);
            relu_mask(r1g, sB, c, acc[nt][2], acc[nt][3], a2, a3);
            const uint32_t top = pack_bf16(a0, a1), bot = pack_bf16(a2, a3);
            *reinterpret_cast<uint32_t *>(dz1 + g * LDH + c) = top;
            *reinterpret_cast<uint32_t *>(dz1 + (g + 8) * LDH + c) = bot;
            if (sA < n) *reinterpret_cast<uint32_t *>(dz1g + sA * H + c) = top;
            if (sB < n) *reinterpret_cast<uint32_t *>(dz1g + sB * H + c) = bot;
        }
    }
    __syncwarp();
    {
        float acc[1][4] = {};
        warp_mma<1>(acc, dz1, LDH, W1T, LDH, H);
        const int c = 2 * t;
        if (sA < n) {
            if (c < D.nA) gin[sA * d + D.A[c]] += acc[0][0];
            if (c + 1 < D.nA) gin[sA * d + D.A[c + 1]] += acc[0][1];
        }
        if (sB < n) {
            if (c < D.nA) gin[sB * d + D.A[c]] += acc[0][2];
            if (c + 1 < D.nA) gin[sB * d + D.A[c + 1]] += acc[0][3];
        }
    }
}

template <int H>
size_t mlp_bwd_data_smem(const LayerDesc &D)
{
    constexpr int LDH = H + 8;
    const int LDO = D.nout_p + 8;
    return sizeof(__nv_bfloat16) * ((size_t)H * LDO + (size_t)H * LDH + 8 * LDH + kTileRows * LDO + kTileRows * LDH);
}

// Weight gradients, split over chunks of 64 samples (persistent CTAs, H/8 warps):
// dW3 = sum_s dL/do[s]^T r2[s], dW2 = sum_s dz2[s]^T r1[s], dW1 = sum_s dz1[s]^T a[s], and the
// bias sums. Each warp keeps its own output tiles in registers across chunks; the CTA adds them
// to the FP32 gradient with atomics once at the end.
template <int H>
__global__ void __launch_bounds__(H * 4) mlp_bwd_weights_kernel(const LayerDesc D, const float *__restrict__ dodraw,
                                                                const __nv_bfloat16 *__restrict__ r1g,
                                                                const __nv_bfloat16 *__restrict__ r2g,
                                                                const __nv_bfloat16 *__restrict__ dz1g,
                                                                const __nv_bfloat16 *__restrict__ dz2g,
                                                                const float *__restrict__ h, int d, long long n,
                                                                float *__restrict__ grad)
{
    constexpr int KC = kTileRows, LDK = KC + 8;
    constexpr int NW = H / 8;                     // warps
    constexpr int MAXT = 24;                      // output tiles per warp (16 x 8 each)
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *gOT = reinterpret_cast<__nv_bfloat16 *>(sm);    // [nout_p][LDK]
    __nv_bfloat16 *r2T = gOT + D.nout_p * LDK;                      // [H][LDK]
    __nv_bfloat16 *r1T = r2T + H * LDK;
    __nv_bfloat16 *dz2T = r1T + H * LDK;
    __nv_bfloat16 *dz1T = dz2T + H * LDK;
    __nv_bfloat16 *aT = dz1T + H * LDK;                               // [8][LDK]

    // output tiles: dW3 (nout_p/16 x H/8), dW2 (H/16 x H/8), dW1 (H/16 x 1)
    const int t3 = (D.nout_p / 16) * (H / 8), t2 = (H / 16) * (H / 8), t1 = H / 16;
    const int ntiles = t3 + t2 + t1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[MAXT][4];
#pragma unroll
    for (int i = 0; i < MAXT; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    constexpr int MAXB = 4;
    float bacc[MAXB] = {0.f, 0.f, 0.f, 0.f};   // bias sums: element threadIdx.x + j blockDim of (b3 | b2 | b1)
    const int nb = D.nout + 2 * H;

    const long long nchunks = (n + KC - 1) / KC;
    for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long long s0 = ch * KC;
        __syncthreads();
        for (int e = threadIdx.x; e < KC * D.nout_p; e += blockDim.x) {
            const int r = e / D.nout_p, c = e - r * D.nout_p;
            const long long s = s0 + r;
            gOT[c * LDK + r] = __float2bfloat16_rn((s < n && c < D.nout) ? dodraw[s * D.nout + c] : 0.f);
        }
        for (int e = threadIdx.x; e < KC * H; e += blockDim.x) {
            const int r = e / H, c = e - r * H;
            const long long s = s0 + r;
            const bool ok = s < n;
            const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
            r2T[c * LDK + r] = ok ? r2g[s * H + c] : z;
            r1T[c * LDK + r] = ok ? r1g[s * H + c] : z;
            dz2T[c * LDK + r] = ok ? dz2g[s * H + c] : z;
            dz1T[c * LDK + r] = ok ? dz1g[s * H + c] : z;
        }
        for (int e = threadIdx.x; e < KC * 8; e += blockDim.x) {
            const int r = e / 8, c = e - r * 8;
            const long long s = s0 + r;
            aT[c * LDK + r] = __float2bfloat16_rn((s < n && c < D.nA) ? h[s * d + D.A[c]] : 0.f);
        }
        __syncthreads();
        // bias sums (dL/do in FP32, dz2 and dz1 as the bf16 values the GEMMs see)
#pragma unroll
        for (int j = 0; j < MAXB; ++j) {
            const int i = threadIdx.x + j * blockDim.x;
            if (i < nb) {
                float sum = 0.f;
                for (int r = 0; r < KC; ++r) {
                    const long long s = s0 + r;
                    if (s >= n) break;
                    if (i < D.nout) sum += dodraw[s * D.nout + i];
                    else if (i < D.nout + H) sum += __bfloat162float(dz2g[s * H + (i - D.nout)]);
                    else sum += __bfloat162float(dz1g[s * H + (i - D.nout - H)]);
                }
                bacc[j] += sum;
            }
        }
#pragma unroll
        for (int slot = 0; slot < MAXT; ++slot) {
            const int tile = warp + slot * NW;
            if (tile >= ntiles) break;
            const __nv_bfloat16 *A, *BT;
            int lda = LDK, ldb = LDK;
            if (tile < t3) {
                const int mt = tile / (H / 8), nt = tile % (H / 8);
                A = gOT + mt * 16 * LDK;
                BT = r2T + nt * 8 * LDK;
            } else if (tile < t3 + t2) {
                const int u = tile - t3, mt = u / (H / 8), nt = u % (H / 8);
                A = dz2T + mt * 16 * LDK;
                BT = r1T + nt * 8 * LDK;
            } else {
                const int mt = tile - t3 - t2;
                A = dz1T + mt * 16 * LDK;
                BT = aT;
            }
            float one[1][4] = {{acc[slot][0], acc[slot][1], acc[slot][2], acc[slot][3]}};
            warp_mma<1>(one, A, lda, BT, ldb, KC);
            acc[slot][0] = one[0][0]; acc[slot][1] = one[0][1]; acc[slot][2] = one[0][2]; acc[slot][3] = one[0][3];
        }
    }
    // flush
#pragma unroll
    for (int slot = 0; slot < MAXT; ++slot) {
        const int tile = warp + slot * NW;
        if (tile >= ntiles) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = g + (q >= 2 ? 8 : 0), col = 2 * t + (q & 1);
            long long idx = -1;
            if (tile < t3) {
                const int mt = tile / (H / 8), nt = tile % (H / 8);
                const int o = mt * 16 + row, hcol = nt * 8 + col;
                if (o < D.nout) idx = D.offW3 + (long long)o * H + hcol;
            } else if (tile < t3 + t2) {
                const int u = tile - t3, mt = u / (H / 8), nt = u % (H / 8);
                idx = D.offW2 + (long long)(mt * 16 + row) * H + nt * 8 + col;
            } else {
                const int mt = tile - t3 - t2;
                if (col < D.nA) idx = D.offW1 + (long long)(mt * 16 + row) * D.nA + col;
            }
            if (idx >= 0 && acc[slot][q] != 0.f) atomicAdd(&grad[idx], acc[slot][q]);
        }
    }
#pragma unroll
    for (int j = 0; j < MAXB; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < nb && bacc[j] != 0.f) {
            long long idx;
            if (i < D.nout) idx = D.offb3 + i;
            else if (i < D.nout + H) idx = D.offb2 + (i - D.nout);
            else idx = D.offb1 + (i - D.nout - H);
            atomicAdd(&grad[idx], bacc[j]);
        }
    }
}

template <int H>
size_t mlp_bwd_weights_smem(const LayerDesc &D)
{
    constexpr int LDK = kTileRows + 8;
    return sizeof(__nv_bfloat16) * ((size_t)D.nout_p * LDK + 4 * (size_t)H * LDK + 8 * LDK);
}

// ------------------------------------------------------------------------------ loss, Adam
// variance (chi^2): L = sum w e^{-log q}, dL/dlogq = -w e^{-log q}; KL: L = -sum w log q, dL/dlogq = -w.
__global__ void loss_kernel(const float *__restrict__ logq, const float *__restrict__ w, long long n, int kind,
                            float *__restrict__ gl, float *__restrict__ loss)
{
    float local = 0.f;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        float l, gg;
        if (kind == 0) {
            const float e = w[s] * __expf(-logq[s]);
            l = e;
            gg = -e;
        } else {
            l = -w[s] * logq[s];
            gg = -w[s];
        }
        gl[s] = gg;
        local += l;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, local);
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m,
                            float *__restrict__ v, long long np, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        const float gg = gr[i];
        const float mm = b1 * m[i] + (1.f - b1) * gg;
        const float vv = b2 * v[i] + (1.f - b2) * gg * gg;
        m[i] = mm;
        v[i] = vv;
        p[i] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// ------------------------------------------------------------------------------ host side
template <int H>
int mlp_fwd(const float *params, const LayerDesc &D, const float *h, int d, long long n, float *o,
            __nv_bfloat16 *r1, __nv_bfloat16 *r2, cudaStream_t s)
{
    const size_t smem = mlp_fwd_smem<H>(D);
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const long long blocks = (n + kTileRows - 1) / kTileRows;
    mlp_fwd_kernel<H><<<(unsigned)blocks, 128, smem, s>>>(params, D, h, d, n, o, r1, r2);
    return (int)cudaGetLastError();
}

template <int H>
int mlp_bwd(const float *params, const LayerDesc &D, const float *dodraw, const __nv_bfloat16 *r1,
            const __nv_bfloat16 *r2, long long n, int d, __nv_bfloat16 *dz1, __nv_bfloat16 *dz2, float *gin,
            const float *h, float *grad, int num_sms, cudaStream_t s)
{
    size_t smem = mlp_bwd_data_smem<H>(D);
    cudaError_t e = cudaFuncSetAttribute(mlp_bwd_data_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const long long blocks = (n + kTileRows - 1) / kTileRows;
    mlp_bwd_data_kernel<H><<<(unsigned)blocks, 128, smem, s>>>(params, D, dodraw, r1, r2, n, d, dz1, dz2, gin);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    {   // register capacity of the weight-gradient kernel: 24 output tiles per warp, 4 bias sums per thread
        const int ntiles = (D.nout_p / 16) * (H / 8) + (H / 16) * (H / 8) + H / 16;
        if ((ntiles + H / 8 - 1) / (H / 8) > 24 || D.nout + 2 * H > 4 * H * 4) return (int)cudaErrorInvalidConfiguration;
    }
    smem = mlp_bwd_weights_smem<H>(D);
    e = cudaFuncSetAttribute(mlp_bwd_weights_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    long long wb = (n + kTileRows - 1) / kTileRows;
    if (wb > (long long)num_sms * 2) wb = (long long)num_sms * 2;
    mlp_bwd_weights_kernel<H><<<(unsigned)wb, H * 4, smem, s>>>(D, dodraw, r1, r2, dz1, dz2, h, d, n, grad);
    return (int)cudaGetLastError();
}

inline int dispatch_fwd(const Shape &S, const float *params, const LayerDesc &D, const float *h, long long n, float *o,
                        __nv_bfloat16 *r1, __nv_bfloat16 *r2, cudaStream_t s)
{
    switch (S.H) {
    case 32: return mlp_fwd<32>(params, D, h, S.d, n, o, r1, r2, s);
    case 64: return mlp_fwd<64>(params, D, h, S.d, n, o, r1, r2, s);
    default: return mlp_fwd<128>(params, D, h, S.d, n, o, r1, r2, s);
    }
}

inline int dispatch_bwd(const Shape &S, const float *params, const LayerDesc &D, const float *dodraw,
                        const __nv_bfloat16 *r1, const __nv_bfloat16 *r2, long long n, __nv_bfloat16 *dz1,
                        __nv_bfloat16 *dz2, float *gin, const float *h, float *grad, int sms, cudaStream_t s)
{
    switch (S.H) {
    case 32: return mlp_bwd<32>(params, D, dodraw, r1, r2, n, S.d, dz1, dz2, gin, h, grad, sms, s);
    case 64: return mlp_bwd<64>(params, D, dodraw, r1, r2, n, S.d, dz1, dz2, gin, h, grad, sms, s);
    default: return mlp_bwd<128>(params, D, dodraw, r1, r2, n, S.d, dz1, dz2, gin, h, grad, sms, s);
    }
}

inline int launch_coupling(const Shape &S, const LayerDesc &D, const float *o, const float *hin, float *hout,
                           float *logq, long long n, int mode, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n + 255) / 256, 65535);
    switch (S.K) {
    case 4: coupling_kernel<4><<<(unsigned)blocks, 256, 0, s>>>(D, o, hin, hout, logq, S.d, n, mode); break;
    case 8: coupling_kernel<8><<<(unsigned)blocks, 256, 0, s>>>(D, o, hin, hout, logq, S.d, n, mode); break;
    case 16: coupling_kernel<16><<<(unsigned)blocks, 256, 0, s>>>(D, o, hin, hout, logq, S.d, n, mode); break;
    default: coupling_kernel<32><<<(unsigned)blocks, 256, 0, s>>>(D, o, hin, hout, logq, S.d, n, mode); break;
    }
    return (int)cudaGetLastError();
}

inline int launch_coupling_bwd(const Shape &S, const LayerDesc &D, const float *o, const float *hin, const float *gout,
                               const float *gl, float *dodraw, float *gin, long long n, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n + 127) / 128, 65535);
    switch (S.K) {
    case 4: coupling_bwd_kernel<4><<<(unsigned)blocks, 128, 0, s>>>(D, o, hin, gout, gl, dodraw, gin, S.d, n); break;
    case 8: coupling_bwd_kernel<8><<<(unsigned)blocks, 128, 0, s>>>(D, o, hin, gout, gl, dodraw, gin, S.d, n); break;
    case 16: coupling_bwd_kernel<16><<<(unsigned)blocks, 128, 0, s>>>(D, o, hin, gout, gl, dodraw, gin, S.d, n); break;
    default: coupling_bwd_kernel<32><<<(unsigned)blocks, 128, 0, s>>>(D, o, hin, gout, gl, dodraw, gin, S.d, n); break;
    }
    return (int)cudaGetLastError();
}

// Workspace of n samples: h_0..h_L (L+1) x n x d | o, dL/do n x nout_max | r1, r2, dz1, dz2 n x H
// (bf16) | gA, gB n x d | logq, gl n.
struct Work {
    float *hs, *o, *dO, *gA, *gB, *logq, *gl;
    __nv_bfloat16 *r1, *r2, *dz1, *dz2;
    float *part;               // fused training: per-block partial gradients
    long long part_stride;
    int part_rows;
    unsigned char *mirror;     // fused kernels: the bf16 weight mirror
    size_t mirror_bytes;
    int *err;                  // tcgen05 training: bounded-wait error word
};

// Fused training scratch for n samples: the mirror and the partial-gradient rows (one per
// backward block, at most kFusedPartRowsMax, each as long as the largest layer).
inline void fused_extent(const Shape &S, long long n, size_t &mirror_bytes, long long &stride, int &rows)
{
    FusedFlow F;
    mirror_bytes = 0;
    stride = 0;
    rows = 0;
    if (!fused_layout(S, F)) return;
    mirror_bytes = F.total_bytes;
    long long pos = 0, big = 0;
    for (int l = 0; l < S.L; ++l) {
        const long long p0 = pos;
        describe(S, l, pos);
        big = std::max(big, pos - p0);
    }
    stride = (big + 63) / 64 * 64;
    rows = (int)std::min<long long>((n + kFusedBwdRows - 1) / kFusedBwdRows, kFusedPartRowsMax);
}

inline size_t work_bytes(const Shape &S, long long n, int &nout_max)
{
    nout_max = 0;
    long long pos = 0;
    for (int l = 0; l < S.L; ++l) nout_max = std::max(nout_max, describe(S, l, pos).nout);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t mb;
    long long stride;
    int rows;
    fused_extent(S, n, mb, stride, rows);
    return al(sizeof(float) * (size_t)(S.L + 1) * n * S.d) + 2 * al(sizeof(float) * (size_t)n * nout_max) +
           4 * al(sizeof(__nv_bfloat16) * (size_t)n * S.H) + 2 * al(sizeof(float) * (size_t)n * S.d) +
           2 * al(sizeof(float) * (size_t)n) + al(mb) + al(sizeof(float) * (size_t)stride * rows) + al(sizeof(int));
}

inline Work carve(const Shape &S, long long n, void *base)
{
    int nout_max;
    work_bytes(S, n, nout_max);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *q = (char *)base;
    Work w;
    w.hs = (float *)q; q += al(sizeof(float) * (size_t)(S.L + 1) * n * S.d);
    w.o = (float *)q; q += al(sizeof(float) * (size_t)n * nout_max);
    w.dO = (float *)q; q += al(sizeof(float) * (size_t)n * nout_max);
    w.r1 = (__nv_bfloat16 *)q; q += al(sizeof(__nv_bfloat16) * (size_t)n * S.H);
    w.r2 = (__nv_bfloat16 *)q; q += al(sizeof(__nv_bfloat16) * (size_t)n * S.H);
    w.dz1 = (__nv_bfloat16 *)q; q += al(sizeof(__nv_bfloat16) * (size_t)n * S.H);
    w.dz2 = (__nv_bfloat16 *)q; q += al(sizeof(__nv_bfloat16) * (size_t)n * S.H);
    w.gA = (float *)q; q += al(sizeof(float) * (size_t)n * S.d);
    w.gB = (float *)q; q += al(sizeof(float) * (size_t)n * S.d);
    w.logq = (float *)q; q += al(sizeof(float) * (size_t)n);
    w.gl = (float *)q; q += al(sizeof(float) * (size_t)n);
    size_t mb;
    fused_extent(S, n, mb, w.part_stride, w.part_rows);
    w.mirror = (unsigned char *)q; q += al(mb);
    w.mirror_bytes = mb;
    w.part = (float *)q; q += al(sizeof(float) * (size_t)w.part_stride * w.part_rows);
    w.err = (int *)q;
    return w;
}

// Density direction: x -> z, log q. Uses w.hs for the per-layer inputs when keep is set
// (h_l at w.hs + l n d), else ping-pongs between w.gA and w.gB.
inline int run_forward(const Shape &S, const float *params, long long n, const float *x, float *z, float *logq,
                       Work &w, bool keep, cudaStream_t s)
{
    int st = (int)cudaMemsetAsync(logq, 0, sizeof(float) * n, s);
    if (st) return st;
    const size_t nd = (size_t)n * S.d;
    const float *cur = x;
    long long pos = 0;
    if (keep) {
        st = (int)cudaMemcpyAsync(w.hs, x, sizeof(float) * nd, cudaMemcpyDeviceToDevice, s);
        if (st) return st;
        cur = w.hs;
    }
    for (int l = 0; l < S.L; ++l) {
        const LayerDesc D = describe(S, l, pos);
        if ((st = dispatch_fwd(S, params, D, cur, n, w.o, nullptr, nullptr, s))) return st;
        float *next = keep ? w.hs + (size_t)(l + 1) * nd : ((l == S.L - 1) ? z : (l % 2 == 0 ? w.gA : w.gB));
        if ((st = launch_coupling(S, D, w.o, cur, next, logq, n, 0, s))) return st;
        cur = next;
    }
    if (keep) st = (int)cudaMemcpyAsync(z, cur, sizeof(float) * nd, cudaMemcpyDeviceToDevice, s);
    return st;
}

inline int run_inverse(const Shape &S, const float *params, long long n, const float *z, float *x, float *logq,
                       Work &w, cudaStream_t s)
{
    int st = (int)cudaMemsetAsync(logq, 0, sizeof(float) * n, s);
    if (st) return st;
    std::vector<LayerDesc> Ds;
    long long pos = 0;
    for (int l = 0; l < S.L; ++l) Ds.push_back(describe(S, l, pos));
    const float *cur = z;
    for (int l = S.L - 1, k = 0; l >= 0; --l, ++k) {
        if ((st = dispatch_fwd(S, params, Ds[l], cur, n, w.o, nullptr, nullptr, s))) return st;
        float *next = (l == 0) ? x : (k % 2 == 0 ? w.gA : w.gB);
        if ((st = launch_coupling(S, Ds[l], w.o, cur, next, logq, n, 1, s))) return st;
        cur = next;
    }
    return st;
}

// One gradient evaluation: forward with kept activations, loss gradient, then each layer's
// backward from the last to the first. grad and loss accumulate.
inline int run_grad(const Shape &S, const float *params, long long n, const float *x, const float *wts, int kind,
                    float *grad, float *loss, Work &w, int sms, cudaStream_t s)
{
    int st = run_forward(S, params, n, x, w.gB, w.logq, w, true, s);
    if (st) return st;
    const long long lb = std::min<long long>((n + 255) / 256, 4096);
    loss_kernel<<<(unsigned)lb, 256, 0, s>>>(w.logq, wts, n, kind, w.gl, loss);
    if ((st = (int)cudaGetLastError())) return st;
    const size_t nd = (size_t)n * S.d;
    if ((st = (int)cudaMemsetAsync(w.gA, 0, sizeof(float) * nd, s))) return st;   // dL/dz = 0
    std::vector<LayerDesc> Ds;
    long long pos = 0;
    for (int l = 0; l < S.L; ++l) Ds.push_back(describe(S, l, pos));
    float *gout = w.gA, *gin = w.gB;
    for (int l = S.L - 1; l >= 0; --l) {
        const float *hin = w.hs + (size_t)l * nd;
        if ((st = dispatch_fwd(S, params, Ds[l], hin, n, w.o, w.r1, w.r2, s))) return st;
        if ((st = launch_coupling_bwd(S, Ds[l], w.o, hin, gout, w.gl, w.dO, gin, n, s))) return st;
        if ((st = dispatch_bwd(S, params, Ds[l], w.dO, w.r1, w.r2, n, w.dz1, w.dz2, gin, hin, grad, sms, s))) return st;
        std::swap(gout, gin);
    }
    return MCUBES_OK;
}

inline int sms_of_device()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

}  // namespace flow
}  // namespace mcubes

using namespace mcubes;

namespace {

bool to_shape(const mcubes_flow_shape *p, flow::Shape &S)
{
    if (!p) return false;
    S = flow::Shape{p->d, p->layers, p->hidden, p->bins};
    return flow::shape_ok(S);
}

}  // namespace

extern "C" {

int64_t mcubes_flow_param_count(const mcubes_flow_shape *shape)
{
    flow::Shape S;
    if (!to_shape(shape, S)) return 0;
    return flow::param_count(S);
}

size_t mcubes_flow_work_bytes(const mcubes_flow_shape *shape, int64_t n)
{
    flow::Shape S;
    if (!to_shape(shape, S) || n < 1) return 0;
    int nm;
    return flow::work_bytes(S, n, nm);
}

int mcubes_flow_forward_dev(const mcubes_flow_shape *shape, const float *d_params, int64_t n, const float *d_x,
                            float *d_z, float *d_logq, void *d_work, size_t work_bytes, void *stream)
{
    flow::Shape S;
    if (!to_shape(shape, S)) return MCUBES_ERR_INVALID_ARG;
    if (n < 1 || !d_params || !d_x || !d_z || !d_logq) return MCUBES_ERR_INVALID_ARG;
    int nm;
    if (!d_work || work_bytes < flow::work_bytes(S, n, nm) || ((uintptr_t)d_work & 255u)) return MCUBES_ERR_WORKSPACE;
    flow::Work w = flow::carve(S, n, d_work);
    return cuda_status((cudaError_t)flow::run_forward(S, d_params, n, d_x, d_z, d_logq, w, false, (cudaStream_t)stream));
}

int mcubes_flow_inverse_dev(const mcubes_flow_shape *shape, const float *d_params, int64_t n, const float *d_z,
                            float *d_x, float *d_logq, void *d_work, size_t work_bytes, void *stream)
{
    flow::Shape S;
    if (!to_shape(shape, S)) return MCUBES_ERR_INVALID_ARG;
    if (n < 1 || !d_params || !d_x || !d_z || !d_logq) return MCUBES_ERR_INVALID_ARG;
    int nm;
    if (!d_work || work_bytes < flow::work_bytes(S, n, nm) || ((uintptr_t)d_work & 255u)) return MCUBES_ERR_WORKSPACE;
    flow::Work w = flow::carve(S, n, d_work);
    return cuda_status((cudaError_t)flow::run_inverse(S, d_params, n, d_z, d_x, d_logq, w, (cudaStream_t)stream));
}

int mcubes_flow_grad_dev(const mcubes_flow_shape *shape, const float *d_params, int64_t n, const float *d_x,
                         const float *d_w, int loss_kind, float *d_grad, float *d_loss, void *d_work,
                         size_t work_bytes, void *stream)
{
    flow::Shape S;
    if (!to_shape(shape, S)) return MCUBES_ERR_INVALID_ARG;
    if (n < 1 || !d_params || !d_x || !d_w || !d_grad || (loss_kind != 0 && loss_kind != 1)) return MCUBES_ERR_INVALID_ARG;
    int nm;
    if (!d_work || work_bytes < flow::work_bytes(S, n, nm) || ((uintptr_t)d_work & 255u)) return MCUBES_ERR_WORKSPACE;
    flow::Work w = flow::carve(S, n, d_work);
    flow::FusedFlow F;
    // MCUBES_FLOW_TRAIN selects a path for comparisons: "mma" (fused mma.sync kernels), "chain"
    // (per-layer kernels); by default the tcgen05 kernels where the shape fits them, then the
    // fused mma.sync kernels, then the per-layer chain
    const char *path = std::getenv("MCUBES_FLOW_TRAIN");
    const bool want_tc = !path || (std::strcmp(path, "mma") != 0 && std::strcmp(path, "chain") != 0);
    const bool want_fused = !path || std::strcmp(path, "chain") != 0;
    if (w.part_rows > 0 && flow::fused_layout(S, F)) {
        const flow::FusedTrainWork W{w.hs, w.gA, w.gB, w.gl, w.part, w.part_stride, w.part_rows, w.mirror, w.err};
        if (want_tc) {
            const int st = flow::tc_grad(S, d_params, n, d_x, d_w, loss_kind, d_grad, d_loss, W, w.mirror_bytes,
                                         (cudaStream_t)stream);
            if (st != flow::kFusedUnsupported) return st;
        }
        if (want_fused) {
            const int st = flow::fused_grad(F, d_params, n, S.d, d_x, d_w, loss_kind, d_grad, d_loss, W,
                                            (cudaStream_t)stream);
            if (st != flow::kFusedUnsupported) return st;
        }
    }
    const int sms = flow::sms_of_device();
    if (sms <= 0) return cuda_status(cudaErrorNoDevice);
    return cuda_status((cudaError_t)flow::run_grad(S, d_params, n, d_x, d_w, loss_kind, d_grad, d_loss, w, sms,
                                                   (cudaStream_t)stream));
}

int mcubes_flow_adam_dev(int64_t n_params, float *d_params, const float *d_grad, float *d_m, float *d_v, int step,
                         float lr, void *stream)
{
    if (n_params < 1 || !d_params || !d_grad || !d_m || !d_v || step < 1 || !(lr > 0.f)) return MCUBES_ERR_INVALID_ARG;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
    const long long blocks = std::min<long long>((n_params + 255) / 256, 4096);
    flow::adam_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, n_params, lr, b1,
                                                                         b2, eps, c1, c2);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
