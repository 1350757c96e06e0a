// Fused training step of the coupling flow (the gradient of the variance or KL loss over a
// batch of samples), in L + 2 launches instead of the per-layer chains of flow.cu:
//   1. train_fwd_kernel: all layers in the density direction for 128-sample block tiles, each
//      layer's weights copied once per tile from the bf16 mirror; it saves every layer's input,
//      forms log q, the loss and dL/dlog q.
//   2. train_bwd_kernel, once per layer from the last: per 128-sample tile, each warp recomputes
//      its 16 rows' MLP in registers, runs the coupling backward of each (row, axis) pair, and
//      backpropagates through W3, W2 and W1 (mma.sync with ldmatrix.trans operands, so the
//      forward weight layout serves the transposed products). The weight gradients are then
//      block-level GEMMs over the tile's rows (K = 128): dW3 = dO^T r2, dW2 = dz2^T r1,
//      dW1 = dz1^T a, from bf16 slabs in shared memory; bias gradients are FP32 column sums.
//      Each block writes its partial gradient to its own row of a scratch matrix.
//   3. reduce_part_kernel: the rows of that matrix summed into the gradient (fixed order).
// The arithmetic is the per-layer kernels' (bf16 MLP operands, FP32 accumulation, the same
// pq_transform / pq_backward), so the gradient is the exact gradient of the loss up to the bf16
// rounding of the MLP operands.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>

#include "../../include/mcubes.h"
#include "flow_common.cuh"
#include "internal.h"

namespace mcubes {
namespace flow {

namespace {

constexpr int kTSubF = 1, kTRowsF = kFWarps * 16 * kTSubF;   // forward: 128 samples per block tile
constexpr int kTRowsB = kFWarps * 16;                         // backward: 128 samples per block tile
constexpr int kLDA = 8;                                       // row stride of the layer-input slab

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Four 8x8 bf16 matrices, transposed on load: the m16n8k16 A operand from storage S[k][m]
// (rows of m-contiguous elements). Lane i addresses row i % 8 of matrix i / 8.
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const __nv_bfloat16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

// Two 8x8 bf16 matrices, transposed on load: the B operand from storage S[k][n] (rows of
// n-contiguous elements). Lanes 0..15 address rows k = 0..15.
__device__ __forceinline__ void ldsm_x2_t(uint32_t &b0, uint32_t &b1, const __nv_bfloat16 *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(b0), "=r"(b1)
                 : "r"(smem_u32(p)));
}

template <int H, int K>
constexpr int fwd_min_blocks()
{
    return H <= 64 ? 2 : 1;
}

// ------------------------------------------------------------------------------ forward
// Density direction for n samples x (n x d): saves the input of layer l at hsave + l n d, then
// gl = dL/dlog q and loss += L (kind 0, variance: L = sum w e^{-log q}; kind 1, KL: L = -sum w log q).
template <int H, int K>
__global__ void __launch_bounds__(kFThreads, fwd_min_blocks<H, K>())
    train_fwd_kernel(const FusedFlow F, const unsigned char *__restrict__ mirror, const float *__restrict__ x,
                     const float *__restrict__ w, int kind, int d, long long n, float *__restrict__ hsave,
                     float *__restrict__ gl, float *__restrict__ loss)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, OS = SW + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int HS = d | 1;
    unsigned char *wbuf = smem;
    float *hs = reinterpret_cast<float *>(smem + F.max_bytes);
    float *lqs = hs + kTRowsF * HS;
    float *obuf = lqs + kTRowsF;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, row = lane & 15, half = lane >> 4;
    float *ob = obuf + warp * 2 * 16 * OS;
    const long long ntiles = (n + kTRowsF - 1) / kTRowsF;
    float local = 0.f;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long r0 = tile * kTRowsF;
        for (int e = threadIdx.x; e < kTRowsF * d; e += kFThreads) {
            const int r = e / d, a = e - r * d;
            hs[r * HS + a] = (r0 + r < n) ? x[(r0 + r) * d + a] : 0.5f;
        }
        for (int r = threadIdx.x; r < kTRowsF; r += kFThreads) lqs[r] = 0.f;
        for (int l = 0; l < F.L; ++l) {
            const FusedLayer &Y = F.lay[l];
            __syncthreads();   // hs complete; the previous layer is done with the weight buffer
            {
                const uint4 *src = reinterpret_cast<const uint4 *>(mirror + Y.off);
                uint4 *dst = reinterpret_cast<uint4 *>(wbuf);
                for (uint32_t e = threadIdx.x; e < Y.bytes / 16u; e += kFThreads) dst[e] = src[e];
            }
            float *hl = hsave + (size_t)l * (size_t)n * d;
            for (int e = threadIdx.x; e < kTRowsF * d; e += kFThreads) {
                const int r = e / d, a = e - r * d;
                if (r0 + r < n) hl[(r0 + r) * d + a] = hs[r * HS + a];
            }
            __syncthreads();
            for (int sub = 0; sub < kTSubF; ++sub) {
                const int R0 = (warp * kTSubF + sub) * 16;
                const float lq = layer_rows16<H, K>(Y, wbuf, hs, HS, R0, ob, 0);
                if (half == 0) lqs[R0 + row] += lq;
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < kTRowsF; r += kFThreads) {
            const long long s = r0 + r;
            if (s >= n) continue;
            const float lq = lqs[r];
            float lv, gg;
            if (kind == 0) {
                const float e = w[s] * __expf(-lq);
                lv = e;
                gg = -e;
            } else {
                lv = -w[s] * lq;
                gg = -w[s];
            }
            gl[s] = gg;
            local += lv;
        }
        __syncthreads();   // the next tile overwrites hs and lqs
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if (lane == 0 && loss) atomicAdd(loss, local);
}

// ------------------------------------------------------------------------------ backward
// Shared memory of the backward kernel: the layer's weights, the bf16 slabs of a 128-row tile
// (dL/do in slot layout, r1, r2, dz1, dz2, the layer-1 input), the per-warp FP32 slot buffers and
// the FP32 bias-gradient sums.
struct BwdSmem {
    size_t w, dO, r1, r2, dz1, dz2, a, ob, db3, db2, db1, total;
    int ldo;
};

template <int H, int K>
BwdSmem bwd_smem(const FusedFlow &F, int M3p)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, OS = SW + 1, LDH = H + 8;
    BwdSmem B;
    B.ldo = M3p + 8;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += (b + 15) & ~(size_t)15; return r; };
    B.w = take(F.max_bytes);
    B.dO = take(2 * (size_t)kTRowsB * B.ldo);
    B.r1 = take(2 * (size_t)kTRowsB * LDH);
    B.r2 = take(2 * (size_t)kTRowsB * LDH);
    B.dz1 = take(2 * (size_t)kTRowsB * LDH);
    B.dz2 = take(2 * (size_t)kTRowsB * LDH);
    B.a = take(2 * (size_t)kTRowsB * kLDA);
    B.ob = take(4 * (size_t)kFWarps * 2 * 16 * OS);
    B.db3 = take(4 * (size_t)M3p);
    B.db2 = take(4 * (size_t)H);
    B.db1 = take(4 * (size_t)H);
    B.total = o;
    return B;
}

// dL/dh_l for layer l from gout = dL/dh_{l+1} (NULL: zero, the last layer) and gl = dL/dlog q;
// the block's partial gradient of the layer's parameters goes to part + blockIdx.x * pstride
// (layer-local parameter order).
template <int H, int K>
__global__ void __launch_bounds__(kFThreads, 1)
    train_bwd_kernel(const FusedFlow F, const unsigned char *__restrict__ mirror, int l, const BwdSmem SM,
                     const float *__restrict__ hin, const float *__restrict__ gout, const float *__restrict__ gl,
                     float *__restrict__ gin, int d, long long n, float *__restrict__ part, long long pstride)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, OS = SW + 1, NO = 2 * K + 1, LD0 = kK0 + 8, LDH = H + 8;
    extern __shared__ __align__(16) unsigned char smem[];
    const FusedLayer &Y = F.lay[l];
    const int nB = Y.nB, nA = Y.nA, M3 = nB * SW, M3p = round16(M3), LDO = SM.ldo;
    unsigned char *wbuf = smem + SM.w;
    __nv_bfloat16 *dO = reinterpret_cast<__nv_bfloat16 *>(smem + SM.dO);
    __nv_bfloat16 *r1s = reinterpret_cast<__nv_bfloat16 *>(smem + SM.r1);
    __nv_bfloat16 *r2s = reinterpret_cast<__nv_bfloat16 *>(smem + SM.r2);
    __nv_bfloat16 *dz1s = reinterpret_cast<__nv_bfloat16 *>(smem + SM.dz1);
    __nv_bfloat16 *dz2s = reinterpret_cast<__nv_bfloat16 *>(smem + SM.dz2);
    __nv_bfloat16 *as = reinterpret_cast<__nv_bfloat16 *>(smem + SM.a);
    float *obuf = reinterpret_cast<float *>(smem + SM.ob);
    float *db3 = reinterpret_cast<float *>(smem + SM.db3);
    float *db2 = reinterpret_cast<float *>(smem + SM.db2);
    float *db1 = reinterpret_cast<float *>(smem + SM.db1);
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(wbuf);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(wbuf + Y.oW2);
    const __nv_bfloat16 *W3 = reinterpret_cast<const __nv_bfloat16 *>(wbuf + Y.oW3);
    const float *b1 = reinterpret_cast<const float *>(wbuf + Y.ob1);
    const float *b2 = reinterpret_cast<const float *>(wbuf + Y.ob2);
    const float *b3 = reinterpret_cast<const float *>(wbuf + Y.ob3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row = lane & 15, half = lane >> 4;
    float *ob = obuf + warp * 2 * 16 * OS;
    const int R0 = warp * 16;
    // layer-local parameter offsets
    const int pW1 = 0, pb1 = (int)(Y.pb1 - Y.pW1), pW2 = (int)(Y.pW2 - Y.pW1), pb2 = (int)(Y.pb2 - Y.pW1);
    const int pW3 = (int)(Y.pW3 - Y.pW1), pb3 = (int)(Y.pb3 - Y.pW1);
    float *__restrict__ prow = part + (size_t)blockIdx.x * (size_t)pstride;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(mirror + Y.off);
        uint4 *dst = reinterpret_cast<uint4 *>(wbuf);
        for (uint32_t e = threadIdx.x; e < Y.bytes / 16u; e += kFThreads) dst[e] = src[e];
    }
    for (int e = threadIdx.x; e < M3p; e += kFThreads) db3[e] = 0.f;
    for (int e = threadIdx.x; e < H; e += kFThreads) {
        db2[e] = 0.f;
        db1[e] = 0.f;
    }
    // the slab columns between the last slot and the 16-aligned width stay zero
    for (int e = threadIdx.x; e < kTRowsB * (M3p - M3); e += kFThreads) {
        const int r = e / (M3p - M3), c = M3 + e % (M3p - M3);
        dO[r * LDO + c] = __float2bfloat16_rn(0.f);
    }
    __syncthreads();

    const long long ntiles = (n + kTRowsB - 1) / kTRowsB;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const bool first = tile == blockIdx.x;
        const long long base = tile * kTRowsB;
        const long long sg = base + R0 + g, sg8 = sg + 8, sr = base + R0 + row;
        // ---- per warp: recompute the MLP of rows R0..R0+15
        const int xA0 = 2 * t < nA ? Y.A[2 * t] : -1, xA1 = 2 * t + 1 < nA ? Y.A[2 * t + 1] : -1;
        uint32_t a1[4];
        {
            const float v0 = (sg < n && xA0 >= 0) ? hin[sg * d + xA0] : 0.f;
            const float v1 = (sg < n && xA1 >= 0) ? hin[sg * d + xA1] : 0.f;
            const float v2 = (sg8 < n && xA0 >= 0) ? hin[sg8 * d + xA0] : 0.f;
            const float v3 = (sg8 < n && xA1 >= 0) ? hin[sg8 * d + xA1] : 0.f;
            a1[0] = pack_bf16(v0, v1);
            a1[1] = pack_bf16(v2, v3);
            a1[2] = 0u;
            a1[3] = 0u;
            *reinterpret_cast<uint32_t *>(as + (R0 + g) * kLDA + 2 * t) = a1[0];
            *reinterpret_cast<uint32_t *>(as + (R0 + g + 8) * kLDA + 2 * t) = a1[1];
        }
        uint32_t a2[H / 16][4], a3[H / 16][4];
        {
            float acc[H / 8][4] = {};
#pragma unroll
            for (int nt = 0; nt < H / 8; ++nt) {
                const __nv_bfloat16 *bp = W1 + (nt * 8 + g) * LD0 + 2 * t;
                mma16816(acc[nt], a1, ld32(bp), ld32(bp + 8));
            }
            relu_to_operand<H>(acc, b1, a2);
        }
        {
            float acc[H / 8][4] = {};
#pragma unroll
            for (int kt = 0; kt < H / 16; ++kt)
#pragma unroll
                for (int nt = 0; nt < H / 8; ++nt) {
                    const __nv_bfloat16 *bp = W2 + (nt * 8 + g) * LDH + kt * 16 + 2 * t;
                    mma16816(acc[nt], a2[kt], ld32(bp), ld32(bp + 8));
                }
            relu_to_operand<H>(acc, b2, a3);
        }
#pragma unroll
        for (int kt = 0; kt < H / 16; ++kt) {
            const int c = 16 * kt + 2 * t;
            *reinterpret_cast<uint32_t *>(r1s + (R0 + g) * LDH + c) = a2[kt][0];
            *reinterpret_cast<uint32_t *>(r1s + (R0 + g + 8) * LDH + c) = a2[kt][1];
            *reinterpret_cast<uint32_t *>(r1s + (R0 + g) * LDH + c + 8) = a2[kt][2];
            *reinterpret_cast<uint32_t *>(r1s + (R0 + g + 8) * LDH + c + 8) = a2[kt][3];
            *reinterpret_cast<uint32_t *>(r2s + (R0 + g) * LDH + c) = a3[kt][0];
            *reinterpret_cast<uint32_t *>(r2s + (R0 + g + 8) * LDH + c) = a3[kt][1];
            *reinterpret_cast<uint32_t *>(r2s + (R0 + g) * LDH + c + 8) = a3[kt][2];
            *reinterpret_cast<uint32_t *>(r2s + (R0 + g + 8) * LDH + c + 8) = a3[kt][3];
        }
        // ---- coupling backward, two output slots at a time: dL/do into the dO slab (bf16) and
        // the bias sums (FP32); dL/dx of the B axes straight to gin
        const float glq = sr < n ? gl[sr] : 0.f;
        for (int jp = 0; jp < nB; jp += 2) {
            gemm3_pair<H, K>(W3, b3, a3, nB, jp, ob);
            __syncwarp();
            const int j = jp + half;
            if (j < nB) {
                float *raw = ob + half * 16 * OS + row * OS;
                const int ax = Y.B[j];
                const float xv = sr < n ? hin[sr * d + ax] : 0.5f;
                const float gy = (sr < n && gout) ? gout[sr * d + ax] : 0.f;
                const float gx = pq_backward<K>(raw, xv, gy, glq, [raw](int k, float v) { raw[k] = v; });
                for (int k = NO; k < SW; ++k) raw[k] = 0.f;
                if (sr < n) gin[sr * d + ax] = gx;
            }
            __syncwarp();
            for (int idx = lane; idx < 2 * SW; idx += 32) {
                const int hh = idx / SW, k = idx - hh * SW, j2 = jp + hh;
                if (j2 < nB) {
                    const float *col = ob + hh * 16 * OS + k;
                    float sum = 0.f;
#pragma unroll 4
                    for (int r = 0; r < 16; ++r) {
                        const float v = col[r * OS];
                        sum += v;
                        dO[(R0 + r) * LDO + j2 * SW + k] = __float2bfloat16_rn(v);
                    }
                    if (k < NO) atomicAdd(&db3[j2 * SW + k], sum);
                }
            }
            __syncwarp();
        }
        // ---- dr2 = dO W3 (K = the slot-padded outputs), then dz2 = dr2 where r2 > 0
        uint32_t d2[H / 16][4];
        {
            float acc[H / 8][4] = {};
            for (int ks = 0; ks < M3p / 16; ++ks) {
                uint32_t a[4];
                const __nv_bfloat16 *ap = dO + (R0 + g) * LDO + ks * 16 + 2 * t;
                a[0] = ld32(ap);
                a[1] = ld32(ap + 8 * LDO);
                a[2] = ld32(ap + 8);
                a[3] = ld32(ap + 8 * LDO + 8);
#pragma unroll
                for (int nt = 0; nt < H / 8; ++nt) {
                    uint32_t b0, b1v;
                    ldsm_x2_t(b0, b1v, W3 + (ks * 16 + (lane & 15)) * LDH + nt * 8);
                    mma16816(acc[nt], a, b0, b1v);
                }
            }
            float cs[H / 8][2];
#pragma unroll
            for (int kt = 0; kt < H / 16; ++kt) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int nt = 2 * kt + hh;
                    const uint32_t top = a3[kt][2 * hh], bot = a3[kt][2 * hh + 1];
                    const float v0 = (top & 0x7FFFu) ? acc[nt][0] : 0.f;
                    const float v1 = (top & 0x7FFF0000u) ? acc[nt][1] : 0.f;
                    const float v2 = (bot & 0x7FFFu) ? acc[nt][2] : 0.f;
                    const float v3 = (bot & 0x7FFF0000u) ? acc[nt][3] : 0.f;
                    d2[kt][2 * hh] = pack_bf16(v0, v1);
                    d2[kt][2 * hh + 1] = pack_bf16(v2, v3);
                    cs[nt][0] = v0 + v2;
                    cs[nt][1] = v1 + v3;
                }
                const int c = 16 * kt + 2 * t;
                *reinterpret_cast<uint32_t *>(dz2s + (R0 + g) * LDH + c) = d2[kt][0];
                *reinterpret_cast<uint32_t *>(dz2s + (R0 + g + 8) * LDH + c) = d2[kt][1];
                *reinterpret_cast<uint32_t *>(dz2s + (R0 + g) * LDH + c + 8) = d2[kt][2];
                *reinterpret_cast<uint32_t *>(dz2s + (R0 + g + 8) * LDH + c + 8) = d2[kt][3];
            }
#pragma unroll
            for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float v = cs[nt][u];
                    v += __shfl_xor_sync(0xffffffffu, v, 4);
                    v += __shfl_xor_sync(0xffffffffu, v, 8);
                    v += __shfl_xor_sync(0xffffffffu, v, 16);
                    if (g == 0) atomicAdd(&db2[nt * 8 + 2 * t + u], v);
                }
        }
        // ---- dr1 = dz2 W2, then dz1 = dr1 where r1 > 0
        uint32_t d1[H / 16][4];
        {
            float acc[H / 8][4] = {};
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks)
#pragma unroll
                for (int nt = 0; nt < H / 8; ++nt) {
                    uint32_t b0, b1v;
                    ldsm_x2_t(b0, b1v, W2 + (ks * 16 + (lane & 15)) * LDH + nt * 8);
                    mma16816(acc[nt], d2[ks], b0, b1v);
                }
            float cs[H / 8][2];
#pragma unroll
            for (int kt = 0; kt < H / 16; ++kt) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int nt = 2 * kt + hh;
                    const uint32_t top = a2[kt][2 * hh], bot = a2[kt][2 * hh + 1];
                    const float v0 = (top & 0x7FFFu) ? acc[nt][0] : 0.f;
                    const float v1 = (top & 0x7FFF0000u) ? acc[nt][1] : 0.f;
                    const float v2 = (bot & 0x7FFFu) ? acc[nt][2] : 0.f;
                    const float v3 = (bot & 0x7FFF0000u) ? acc[nt][3] : 0.f;
                    d1[kt][2 * hh] = pack_bf16(v0, v1);
                    d1[kt][2 * hh + 1] = pack_bf16(v2, v3);
                    cs[nt][0] = v0 + v2;
                    cs[nt][1] = v1 + v3;
                }
                const int c = 16 * kt + 2 * t;
                *reinterpret_cast<uint32_t *>(dz1s + (R0 + g) * LDH + c) = d1[kt][0];
                *reinterpret_cast<uint32_t *>(dz1s + (R0 + g + 8) * LDH + c) = d1[kt][1];
                *reinterpret_cast<uint32_t *>(dz1s + (R0 + g) * LDH + c + 8) = d1[kt][2];
                *reinterpret_cast<uint32_t *>(dz1s + (R0 + g + 8) * LDH + c + 8) = d1[kt][3];
            }
#pragma unroll
            for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float v = cs[nt][u];
                    v += __shfl_xor_sync(0xffffffffu, v, 4);
                    v += __shfl_xor_sync(0xffffffffu, v, 8);
                    v += __shfl_xor_sync(0xffffffffu, v, 16);
                    if (g == 0) atomicAdd(&db1[nt * 8 + 2 * t + u], v);
                }
        }
        // ---- da = dz1 W1: dL/dh_l of the A axes (plus their pass-through gradient)
        {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks) {
                uint32_t b0, b1v;
                ldsm_x2_t(b0, b1v, W1 + (ks * 16 + (lane & 15)) * LD0);
                mma16816(acc, d1[ks], b0, b1v);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int c = 2 * t + u;
                if (c < nA) {
                    const int ax = Y.A[c];
                    if (sg < n) gin[sg * d + ax] = (gout ? gout[sg * d + ax] : 0.f) + acc[u];
                    if (sg8 < n) gin[sg8 * d + ax] = (gout ? gout[sg8 * d + ax] : 0.f) + acc[2 + u];
                }
            }
        }
        __syncthreads();   // every warp's slabs are complete
        // ---- weight gradients over the tile's 128 rows: output tiles dealt round-robin to warps
        const int T3 = (M3p / 16) * (H / 8), T2 = (H / 16) * (H / 8), T1 = H / 16;
        for (int tt = warp; tt < T3 + T2 + T1; tt += kFWarps) {
            const __nv_bfloat16 *As, *Bs;
            int lda, ldb, m0, n0, kind;
            if (tt < T3) {
                m0 = (tt / (H / 8)) * 16; n0 = (tt % (H / 8)) * 8;
                As = dO; lda = LDO; Bs = r2s; ldb = LDH; kind = 3;
            } else if (tt < T3 + T2) {
                const int u = tt - T3;
                m0 = (u / (H / 8)) * 16; n0 = (u % (H / 8)) * 8;
                As = dz2s; lda = LDH; Bs = r1s; ldb = LDH; kind = 2;
            } else {
                m0 = (tt - T3 - T2) * 16; n0 = 0;
                As = dz1s; lda = LDH; Bs = as; ldb = kLDA; kind = 1;
            }
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            const int mi = lane >> 3, ri = lane & 7;
#pragma unroll
            for (int ks = 0; ks < kTRowsB / 16; ++ks) {
                uint32_t a[4], b0, b1v;
                ldsm_x4_t(a, As + (ks * 16 + ri + ((mi & 2) ? 8 : 0)) * lda + m0 + ((mi & 1) ? 8 : 0));
                ldsm_x2_t(b0, b1v, Bs + (ks * 16 + (lane & 15)) * ldb + n0);
                mma16816(acc, a, b0, b1v);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int m = m0 + g + ((u & 2) ? 8 : 0), c = n0 + 2 * t + (u & 1);
                int idx = -1;
                if (kind == 3) {
                    const int j = m / SW, k = m - j * SW;
                    if (j < nB && k < NO) idx = pW3 + (j * NO + k) * H + c;
                } else if (kind == 2) {
                    idx = pW2 + m * H + c;
                } else if (c < nA) {
                    idx = pW1 + m * nA + c;
                }
                if (idx >= 0) {
                    if (first) prow[idx] = acc[u];   // every weight entry is written once per tile
                    else prow[idx] += acc[u];
                }
            }
        }
        __syncthreads();   // the slabs are reused by the next tile
    }
    for (int o = threadIdx.x; o < M3; o += kFThreads) {
        const int j = o / SW, k = o - j * SW;
        if (k < NO) prow[pb3 + j * NO + k] = db3[o];
    }
    for (int h = threadIdx.x; h < H; h += kFThreads) {
        prow[pb2 + h] = db2[h];
        prow[pb1 + h] = db1[h];
    }
}

// grad[e] += sum over the blocks' partial rows. A block takes 32 columns; its 8 warps sum every
// 8th row (coalesced 128-byte reads), then warp 0 adds the 8 partial sums in a fixed order.
__global__ void __launch_bounds__(256) reduce_part_kernel(const float *__restrict__ part, int rows, long long pstride,
                                                          int npl, float *__restrict__ grad)
{
    __shared__ float acc[8][33];
    const int c = threadIdx.x & 31, rg = threadIdx.x >> 5, e = blockIdx.x * 32 + c;
    float s = 0.f;
    if (e < npl)
        for (int r = rg; r < rows; r += 8) s += part[(size_t)r * pstride + e];
    acc[rg][c] = s;
    __syncthreads();
    if (rg == 0 && e < npl) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += acc[k][c];
        grad[e] += t;
    }
}

int max_M3p(const FusedFlow &F)
{
    int m = 0;
    for (int l = 0; l < F.L; ++l) m = std::max(m, round16(F.lay[l].nB * F.SW));
    return m;
}

int device_limits(int &optin, int &sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return cuda_status(e);
}

// Per device and kernel instance: the shared-memory opt-in limit is raised once to the device's
// maximum, and the device's limits are read once (the training loop calls this every step).
struct DeviceInfo {
    int optin = 0, sms = 0;
};

int device_info(DeviceInfo &out)
{
    static DeviceInfo cache[64];
    static std::atomic<uint64_t> known{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 64 && (known.load(std::memory_order_acquire) >> dev & 1u)) {
        out = cache[dev];
        return MCUBES_OK;
    }
    DeviceInfo di;
    if (int st = device_limits(di.optin, di.sms)) return st;
    if (dev < 64) {
        cache[dev] = di;
        known.fetch_or(1ull << dev, std::memory_order_release);
    }
    out = di;
    return MCUBES_OK;
}

template <typename Kern>
int raise_smem_limit(Kern kern, int optin, std::atomic<uint64_t> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 64 && (done.load(std::memory_order_acquire) >> dev & 1u)) return MCUBES_OK;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return cuda_status(e);
    // the opt-in limit covers static and dynamic shared memory
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes)) !=
        cudaSuccess)
        return cuda_status(e);
    if (dev < 64) done.fetch_or(1ull << dev, std::memory_order_release);
    return MCUBES_OK;
}

template <int H, int K>
int grad_hk(const FusedFlow &F, const unsigned char *mirror, long long n, int d, const float *x, const float *w,
            int kind, float *grad, float *loss, const FusedTrainWork &W, cudaStream_t s)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7;
    static std::atomic<uint64_t> fwd_done{0}, bwd_done{0};
    DeviceInfo di;
    int st = device_info(di);
    if (st) return st;
    const int HS = d | 1;
    const size_t fsm = (size_t)F.max_bytes + sizeof(float) * ((size_t)kTRowsF * HS + kTRowsF +
                                                              (size_t)kFWarps * 2 * 16 * (SW + 1));
    const BwdSmem B = bwd_smem<H, K>(F, max_M3p(F));
    if (fsm > (size_t)di.optin || B.total > (size_t)di.optin) return kFusedUnsupported;
    if ((st = raise_smem_limit(train_fwd_kernel<H, K>, di.optin, fwd_done))) return st;
    if ((st = raise_smem_limit(train_bwd_kernel<H, K>, di.optin, bwd_done))) return st;
    // resident forward blocks per SM: shared memory (228 KB an SM, 1 KB reserved a block), then
    // the launch bound's two blocks for H <= 64
    const int per_sm = std::max(1, std::min(fwd_min_blocks<H, K>(), (int)(233472 / (fsm + 1024))));
    const long long ftiles = (n + kTRowsF - 1) / kTRowsF;
    const unsigned fgrid = (unsigned)std::min<long long>(ftiles, (long long)per_sm * di.sms);
    train_fwd_kernel<H, K><<<fgrid, kFThreads, fsm, s>>>(F, mirror, x, w, kind, d, n, W.hs, W.gl, loss);
    if ((st = cuda_status(cudaGetLastError()))) return st;
    const long long btiles = (n + kTRowsB - 1) / kTRowsB;
    const int bgrid = (int)std::min<long long>(btiles, std::min<long long>(di.sms, W.part_rows));
    float *gout = nullptr, *gin = W.gA;
    for (int l = F.L - 1; l >= 0; --l) {
        const FusedLayer &Y = F.lay[l];
        const int npl = (int)(Y.pb3 - Y.pW1) + Y.nB * (2 * K + 1);
        train_bwd_kernel<H, K><<<(unsigned)bgrid, kFThreads, B.total, s>>>(
            F, mirror, l, B, W.hs + (size_t)l * (size_t)n * d, gout, W.gl, gin, d, n, W.part, W.part_stride);
        if ((st = cuda_status(cudaGetLastError()))) return st;
        reduce_part_kernel<<<(unsigned)((npl + 31) / 32), 256, 0, s>>>(W.part, bgrid, W.part_stride, npl,
                                                                       grad + Y.pW1);
        if ((st = cuda_status(cudaGetLastError()))) return st;
        gout = gin;
        gin = (gin == W.gA) ? W.gB : W.gA;
    }
    return MCUBES_OK;
}

template <int H>
int grad_h(const FusedFlow &F, const unsigned char *mirror, long long n, int d, const float *x, const float *w,
           int kind, float *grad, float *loss, const FusedTrainWork &W, cudaStream_t s)
{
    switch (F.K) {
    case 4: return grad_hk<H, 4>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    case 8: return grad_hk<H, 8>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    case 16: return grad_hk<H, 16>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    case 32: return grad_hk<H, 32>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    default: return kFusedUnsupported;
    }
}

}  // namespace

int launch_reduce_part(const float *part, int rows, long long pstride, int npl, float *grad, cudaStream_t s)
{
    if (npl <= 0) return MCUBES_OK;
    reduce_part_kernel<<<(unsigned)((npl + 31) / 32), 256, 0, s>>>(part, rows, pstride, npl, grad);
    return cuda_status(cudaGetLastError());
}

int fused_grad(const FusedFlow &F, const float *params, long long n, int d, const float *x, const float *w, int kind,
               float *grad, float *loss, const FusedTrainWork &W, cudaStream_t s)
{
    if (n <= 0) return MCUBES_OK;
    int st = build_mirror(F, params, W.mirror, s);
    if (st) return st;
    switch (F.H) {
    case 32: return grad_h<32>(F, W.mirror, n, d, x, w, kind, grad, loss, W, s);
    case 64: return grad_h<64>(F, W.mirror, n, d, x, w, kind, grad, loss, W, s);
    case 128: return grad_h<128>(F, W.mirror, n, d, x, w, kind, grad, loss, W, s);
    default: return kFusedUnsupported;
    }
}

}  // namespace flow
}  // namespace mcubes
