// Training step of the coupling flow on the fifth-generation tensor cores (tcgen05, TMEM
// accumulators): the gradient of the variance or KL loss over a batch, in L + 1 launches plus one
// fixed-order reduction per layer, for widths 64 and 128.
//
// 1. train_fwd_tc_kernel: 128-sample tiles (sample row r = TMEM lane r, threads r and r + 128),
//    every layer in the density direction: the three GEMMs of the layer's MLP as tcgen05.mma
//    (bf16 operands in shared memory, FP32 accumulators in TMEM), bias and ReLU from TMEM rows,
//    the coupling CDF of each transformed axis (pq_transform) on the row's outputs read straight
//    from TMEM. It saves every layer's input, forms log q, the loss and dL/dlog q.
// 2. train_bwd_tc_kernel, once per layer from the last: per 128-sample tile it recomputes the MLP
//    (three MMAs), runs the coupling backward of each (row, axis) (pq_backward), and then
//      dR2 = dO W3, dR1 = dZ2 W2, dA = dZ1 W1          (data gradients, M = the tile's rows)
//      dW3 = dO^T R2, dW2 = dZ2^T R1, dW1 = dZ1^T A1   (weight gradients, K = the tile's rows)
//    all as tcgen05.mma reading the buffers already in shared memory: the forward weight layout
//    and the activation slabs serve the transposed products as MN-major operands, so no
//    transposed copies are made. The weight gradients are read from TMEM into the CTA's row of a
//    partial-gradient matrix (its tiles added in order); bias gradients are FP32 column sums.
// 3. reduce_part (flow_train.cu): the rows summed into the gradient in a fixed order.
// The arithmetic is the fused mma.sync kernels' (bf16 MLP operands, FP32 accumulation, the same
// pq_transform / pq_backward), so the gradient is the exact gradient of the loss up to the bf16
// rounding of the MLP operands. Every mbarrier wait is bounded: on expiry a kernel records an
// error in the workspace's error word, waits (bounded) for its copy in flight, and frees its TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>

#include "../../include/mcubes.h"
#include "flow_common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace mcubes {
namespace flow {

namespace {

using namespace tc;

constexpr int kTT = 2 * kTcRows;        // 256 threads: two per sample row
constexpr int kBwdCols = 512;            // TMEM columns of a backward CTA: working [0, 256), dW3 [256, 512)

__device__ __forceinline__ bool all_ok(bool ok) { return __syncthreads_and(ok ? 1 : 0) != 0; }

// generic-proxy shared writes -> visible to the next MMA; TMEM reads done before the next MMA
__device__ __forceinline__ void to_mma()
{
    proxy_fence();
    before_sync();
    __syncthreads();
    after_sync();
}

// Bias + ReLU of TMEM row columns [c0, c1) (a multiple of 8 each) into the bf16 operand row `row` of
// a cols-wide slab.
__device__ __forceinline__ void relu_cols(uint32_t taddr, const float *bias, unsigned char *op, int row, int cols,
                                          int c0, int c1)
{
    for (int c = c0; c < c1; c += 8) {
        float v[8];
        tmem_ld8(taddr + (uint32_t)c, v);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            w[j] = pack_bf16(fmaxf(v[2 * j] + bias[c + 2 * j], 0.f), fmaxf(v[2 * j + 1] + bias[c + 2 * j + 1], 0.f));
        *reinterpret_cast<uint4 *>(op + cm_off(row, c, cols)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// dst[0..8) = v (first) or dst[0..8) += v, as two 16-byte accesses (dst 16-byte aligned).
__device__ __forceinline__ void add8(float *dst, const float (&v)[8], bool first)
{
    float4 *p = reinterpret_cast<float4 *>(dst);
    float4 a = make_float4(v[0], v[1], v[2], v[3]), b = make_float4(v[4], v[5], v[6], v[7]);
    if (!first) {
        const float4 x = p[0], y = p[1];
        a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
        b.x += y.x; b.y += y.y; b.z += y.z; b.w += y.w;
    }
    p[0] = a;
    p[1] = b;
}

// Sum of v over the warp's 32 lanes (rows), added to *dst by lane 0.
__device__ __forceinline__ void col_sum_add(float v, float *dst)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(dst, v);
}

// ------------------------------------------------------------------------------ forward
// Density direction for n samples (x: n x d): saves the input of layer l at hsave + l n d, then
// gl = dL/dlog q and loss += L (kind 0, variance: L = sum w e^{-log q}; kind 1, KL: L = -sum w log q).
// The CTA's layer sequence (step s: layer s mod L of its (s / L)-th tile) takes its weights from
// nbuf buffers by bulk copies, the next step's copy issued while the current step computes.
template <int H, int K>
__global__ void __launch_bounds__(kTT, 1)
    train_fwd_tc_kernel(const TcFlow F, const unsigned char *__restrict__ mirror, const float *__restrict__ x,
                        const float *__restrict__ w, int kind, int d, long long n, float *__restrict__ hsave,
                        float *__restrict__ gl, float *__restrict__ loss, int *__restrict__ err, const int nbuf)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_holder;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t wbar[2];
    __shared__ float lq_half[kTcRows];
    const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kTcRows - 1), half = tid >> 7, HS = d | 1;
    const uint32_t wstride = (F.max_bytes + 1023u) & ~1023u;
    unsigned char *const wbuf0 = smem, *const wbuf1 = smem + wstride;
    unsigned char *A1 = smem + (size_t)nbuf * wstride;            // 128 x 16 bf16
    unsigned char *A2 = A1 + kTcRows * 16 * 2;                     // 128 x H bf16
    float *hs = reinterpret_cast<float *>(A2 + kTcRows * H * 2);   // 128 x HS
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&wbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&wbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    before_sync();
    __syncthreads();
    after_sync();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    float *hr = hs + row * HS;
    float local = 0.f;
    const long long ntiles = (n + kTcRows - 1) / kTcRows;
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long n_steps = my_tiles * F.L;
    uint32_t issued0 = 0u, issued1 = 0u, used0 = 0u, used1 = 0u;   // thread 0: copies issued / waited
    auto issue = [&](long long st) {
        const int b = (int)(st % nbuf);
        const TcLayer &Z = F.lay[(int)(st % F.L)];
        proxy_fence();
        bulk_copy_g2s(b ? wbuf1 : wbuf0, mirror + Z.off, Z.bytes, &wbar[b]);
        if (b) ++issued1; else ++issued0;
    };
    if (tid == 0 && n_steps > 0) issue(0);
    long long step = 0;

    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long r0 = tile * kTcRows, sr = r0 + row;
        const int rows = (int)(n - r0 < (long long)kTcRows ? n - r0 : (long long)kTcRows);
        // the tile's rows are contiguous in x: loaded by all threads, coalesced
        for (int e = tid; e < kTcRows * d; e += kTT) {
            const int r = e / d, a = e - r * d;
            hs[r * HS + a] = r < rows ? x[r0 * d + e] : 0.5f;
        }
        float lq = 0.f;
        for (int l = 0; l < F.L && ok; ++l, ++step) {
            const TcLayer &Y = F.lay[l];
            before_sync();
            __syncthreads();   // hs holds layer l's input; the previous layer's MMAs and reads are done
            after_sync();
            {
                float *hl = hsave + (size_t)l * (size_t)n * d + r0 * d;
                for (int e = tid; e < rows * d; e += kTT) hl[e] = hs[(e / d) * HS + e % d];
            }
            const int b = (int)(step % nbuf);
            if (tid == 0) {
                if (nbuf == 2 && step + 1 < n_steps) issue(step + 1);
                if (nbuf == 1) issue(step);
            }
            if (!all_ok(mbar_wait(&wbar[b], (uint32_t)((step / nbuf) & 1)))) { ok = false; break; }
            if (tid == 0) {
                if (b) ++used1; else ++used0;
            }
            const unsigned char *wbuf = b ? wbuf1 : wbuf0;
            const unsigned char *W1 = wbuf, *W2 = wbuf + Y.oW2, *W3 = wbuf + Y.oW3;
            const float *b1 = reinterpret_cast<const float *>(wbuf + Y.ob1);
            const float *b2 = reinterpret_cast<const float *>(wbuf + Y.ob2);
            const float *b3 = reinterpret_cast<const float *>(wbuf + Y.ob3);
            {
                uint32_t wv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c0 = 8 * half + 2 * j, c1 = c0 + 1;
                    wv[j] = pack_bf16(c0 < Y.nA ? hr[Y.A[c0]] : 0.f, c1 < Y.nA ? hr[Y.A[c1]] : 0.f);
                }
                *reinterpret_cast<uint4 *>(A1 + cm_off(row, 8 * half, 16)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            to_mma();
            if (tid == 0) {
                mma_issue(tmem, A1, W1, 16, H);
                mma_commit(&mbar);
            }
            if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
            phase ^= 1u;
            after_sync();
            relu_cols(lane_base, b1, A2, row, H, half * (H / 2), (half + 1) * (H / 2));
            to_mma();
            if (tid == 0) {
                mma_issue(tmem + H, A2, W2, H, H);
                mma_commit(&mbar);
            }
            if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
            phase ^= 1u;
            after_sync();
            relu_cols(lane_base + H, b2, A2, row, H, half * (H / 2), (half + 1) * (H / 2));
            to_mma();
            if (tid == 0) {
                mma_issue(tmem, A2, W3, H, Y.N3);
                mma_commit(&mbar);
            }
            if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
            phase ^= 1u;
            after_sync();
            for (int j = half; j < Y.nB; j += 2) {
                float raw[SW];
#pragma unroll
                for (int c0 = 0; c0 < SW; c0 += 8) {
                    float v[8];
                    tmem_ld8(lane_base + (uint32_t)(j * SW + c0), v);
#pragma unroll
                    for (int u = 0; u < 8; ++u) raw[c0 + u] = v[u] + b3[j * SW + c0 + u];
                }
                float out, qv;
                pq_transform<K>(raw, hr[Y.B[j]], 0, out, qv);
                hr[Y.B[j]] = out;
                lq += __logf(qv);
            }
        }
        if (!ok) break;
        if (half == 1) lq_half[row] = lq;
        __syncthreads();
        if (half == 0 && sr < n) {
            lq += lq_half[row];
            float lv, gg;
            if (kind == 0) {
                const float e = w[sr] * __expf(-lq);
                lv = e;
                gg = -e;
            } else {
                lv = -w[sr] * lq;
                gg = -w[sr];
            }
            gl[sr] = gg;
            local += lv;
        }
    }
    if (ok) {
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((tid & 31) == 0 && loss) atomicAdd(loss, local);
    }
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        for (; used0 < issued0; ++used0) mbar_wait(&wbar[0], used0 & 1u);
        for (; used1 < issued1; ++used1) mbar_wait(&wbar[1], used1 & 1u);
    }
    before_sync();
    __syncthreads();
    after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// ------------------------------------------------------------------------------ backward
// Shared memory of the backward kernel: the layer's weights, the dL/do slab X (128 x N3 bf16), the
// slabs Y (R1, then dZ1) and Z (R2, then dZ2) (128 x H bf16 each), the layer-1 operand A1 (128 x 16),
// the tile's input rows, dL/dlog q and the FP32 bias-gradient sums. X comes before Y and Z: the
// weight-gradient MMAs read 128 MN rows from X (and H < 128 rows from Y, Z), past a slab's last
// column into the slab after it, never past the CTA's shared memory; those rows of the result are
// not used.
struct BwdTcSmem {
    uint32_t w, x, y, z, a1, hs, gls, db3, db2, db1, total;
};

template <int H>
BwdTcSmem bwd_tc_smem(const TcFlow &F, int d)
{
    int n3 = 0;
    for (int l = 0; l < F.L; ++l) n3 = std::max(n3, F.lay[l].N3);
    BwdTcSmem B;
    uint32_t o = 0;
    auto take = [&](size_t b) { const uint32_t r = o; o += (uint32_t)((b + 127) & ~(size_t)127); return r; };
    B.w = take(F.max_bytes);
    B.x = take(2u * kTcRows * (uint32_t)n3);
    B.y = take(2u * kTcRows * H);
    B.z = take(2u * kTcRows * H);
    B.a1 = take(2u * kTcRows * 16);
    B.hs = take(4u * kTcRows * (uint32_t)(d | 1));
    B.gls = take(4u * kTcRows);
    B.db3 = take(4u * (uint32_t)n3);
    B.db2 = take(4u * H);
    B.db1 = take(4u * H);
    B.total = o;
    return B;
}

// dL/dh_l for layer l from gout = dL/dh_{l+1} (NULL: zero, the last layer) and gl = dL/dlog q; the
// CTA's partial gradient of the layer's parameters goes to part + blockIdx.x * pstride
// (layer-local parameter order).
template <int H, int K>
__global__ void __launch_bounds__(kTT, 1)
    train_bwd_tc_kernel(const TcFlow F, const unsigned char *__restrict__ mirror, int l, const BwdTcSmem SM,
                        const float *__restrict__ hin, const float *__restrict__ gout, const float *__restrict__ gl,
                        float *__restrict__ gin, int d, long long n, float *__restrict__ part, long long pstride,
                        int *__restrict__ err)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, NO = 2 * K + 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_holder;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t wbar;
    const TcLayer &Y = F.lay[l];
    const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kTcRows - 1), half = tid >> 7, HS = d | 1;
    const int nB = Y.nB, nA = Y.nA, N3 = Y.N3, M3 = nB * SW;
    unsigned char *wbuf = smem + SM.w;
    unsigned char *X = smem + SM.x, *Ys = smem + SM.y, *Zs = smem + SM.z, *A1 = smem + SM.a1;
    float *hs = reinterpret_cast<float *>(smem + SM.hs);
    float *gls = reinterpret_cast<float *>(smem + SM.gls);
    float *db3 = reinterpret_cast<float *>(smem + SM.db3);
    float *db2 = reinterpret_cast<float *>(smem + SM.db2);
    float *db1 = reinterpret_cast<float *>(smem + SM.db1);
    const unsigned char *W1 = wbuf, *W2 = wbuf + Y.oW2, *W3 = wbuf + Y.oW3;
    const float *b1 = reinterpret_cast<const float *>(wbuf + Y.ob1);
    const float *b2 = reinterpret_cast<const float *>(wbuf + Y.ob2);
    const float *b3 = reinterpret_cast<const float *>(wbuf + Y.ob3);
    // layer-local parameter offsets
    const int pb1 = (int)(Y.pb1 - Y.pW1), pW2 = (int)(Y.pW2 - Y.pW1), pb2 = (int)(Y.pb2 - Y.pW1);
    const int pW3 = (int)(Y.pW3 - Y.pW1), pb3 = (int)(Y.pb3 - Y.pW1);
    float *__restrict__ prow = part + (size_t)blockIdx.x * (size_t)pstride;
    const int c0h = half * (H / 2), c1h = (half + 1) * (H / 2);   // this thread's half of H columns

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                     "r"(kBwdCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&wbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // the X columns past the layer's slots stay zero; the bias sums start at zero
    for (int e = tid; e < kTcRows * (N3 - M3); e += kTT) {
        const int r = e / (N3 - M3), c = M3 + e % (N3 - M3);
        *reinterpret_cast<__nv_bfloat16 *>(X + cm_off(r, c, N3)) = __float2bfloat16_rn(0.f);
    }
    for (int e = tid; e < N3; e += kTT) db3[e] = 0.f;
    for (int e = tid; e < H; e += kTT) {
        db2[e] = 0.f;
        db1[e] = 0.f;
    }
    before_sync();
    __syncthreads();
    after_sync();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t tb = tmem + lane_off;
    uint32_t phase = 0;
    bool ok = true;
    bool copying = false;
    if (tid == 0) {
        bulk_copy_g2s(wbuf, mirror + Y.off, Y.bytes, &wbar);
        copying = true;
    }
    if (!all_ok(mbar_wait(&wbar, 0))) ok = false;
    if (tid == 0 && ok) copying = false;
    float *hr = hs + row * HS;
    const int nc = (N3 + kTcRows - 1) / kTcRows;   // dW3: M = N3 in chunks of 128 output rows

    const long long ntiles = (n + kTcRows - 1) / kTcRows;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const bool first = tile == blockIdx.x;
        const long long r0 = tile * kTcRows, sr = r0 + row;
        const int rows = (int)(n - r0 < (long long)kTcRows ? n - r0 : (long long)kTcRows);
        const bool live = sr < n;
        // the tile's input rows are contiguous: loaded by all threads, coalesced
        for (int e = tid; e < kTcRows * d; e += kTT) {
            const int r = e / d, a = e - r * d;
            hs[r * HS + a] = r < rows ? hin[r0 * d + e] : 0.5f;
        }
        if (half == 0) gls[row] = live ? gl[sr] : 0.f;
        // dL/dh_{l+1} of this row's axes, fetched now so that the loads overlap the recomputation:
        // this half's transformed axes (j = half, half + 2, ...) and the kept axes c = 8 half .. 8 half + 7
        float gyB[(kMaxAB + 1) / 2], gyA[8];
#pragma unroll
        for (int u = 0; u < (kMaxAB + 1) / 2; ++u) {
            const int j = half + 2 * u;
            gyB[u] = (live && gout && j < nB) ? gout[sr * d + Y.B[j]] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = 8 * half + u;
            gyA[u] = (live && gout && c < nA) ? gout[sr * d + Y.A[c]] : 0.f;
        }
        before_sync();
        __syncthreads();
        after_sync();
        {   // the layer-1 operand: the kept coordinates (each half 8 columns)
            uint32_t wv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = 8 * half + 2 * j, c1 = c0 + 1;
                wv[j] = pack_bf16(c0 < nA ? hr[Y.A[c0]] : 0.f, c1 < nA ? hr[Y.A[c1]] : 0.f);
            }
            *reinterpret_cast<uint4 *>(A1 + cm_off(row, 8 * half, 16)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        // ---- recompute the MLP: D1 -> R1 (Y), D2 -> R2 (Z), D3 = the raw outputs
        to_mma();
        if (tid == 0) {
            mma_issue(tmem, A1, W1, 16, H);
            mma_commit(&mbar);
        }
        if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
        phase ^= 1u;
        after_sync();
        relu_cols(tb, b1, Ys, row, H, c0h, c1h);
        to_mma();
        if (tid == 0) {
            mma_issue(tmem + H, Ys, W2, H, H);
            mma_commit(&mbar);
        }
        if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
        phase ^= 1u;
        after_sync();
        relu_cols(tb + H, b2, Zs, row, H, c0h, c1h);
        to_mma();
        if (tid == 0) {
            mma_issue(tmem, Zs, W3, H, N3);
            mma_commit(&mbar);
        }
        if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
        phase ^= 1u;
        after_sync();
        // ---- coupling backward of this half's axes: dL/do into X (bf16), its column sums into db3,
        // dL/dx of the B axes to gin
        const float glq = gls[row];
#pragma unroll 1
        for (int j = half; j < nB; j += 2) {
            float raw[SW];
#pragma unroll
            for (int c0 = 0; c0 < SW; c0 += 8) {
                float v[8];
                tmem_ld8(tb + (uint32_t)(j * SW + c0), v);
#pragma unroll
                for (int u = 0; u < 8; ++u) raw[c0 + u] = v[u] + b3[j * SW + c0 + u];
            }
            const int ax = Y.B[j];
            float gy = 0.f;
#pragma unroll
            for (int u = 0; u < (kMaxAB + 1) / 2; ++u)
                if (half + 2 * u == j) gy = gyB[u];
            const float gx = pq_backward<K>(raw, hr[ax], gy, glq, [&raw](int k, float v) { raw[k] = v; });
#pragma unroll
            for (int k = 0; k < SW; ++k)
                if (k >= NO || !live) raw[k] = 0.f;
            if (live) gin[sr * d + ax] = gx;
#pragma unroll
            for (int c0 = 0; c0 < SW; c0 += 8) {
                uint32_t wv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) wv[u] = pack_bf16(raw[c0 + 2 * u], raw[c0 + 2 * u + 1]);
                *reinterpret_cast<uint4 *>(X + cm_off(row, j * SW + c0, N3)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            // both halves' warps cover the same 32 rows, so each warp sums its own axes' columns
#pragma unroll
            for (int k = 0; k < NO; ++k) col_sum_add(raw[k], &db3[j * SW + k]);
        }
        // ---- dR2 = dO W3 into [0, H); dW3 = dO^T R2 into [256, 256 + nc H)
        to_mma();
        if (tid == 0) {
            mma_ab(tmem, Opnd{X, N3, false, 0}, Opnd{W3, H, true, 0}, N3, H, false);
            for (int c = 0; c < nc; ++c)
                mma_ab(tmem + 256 + (uint32_t)(c * H), Opnd{X, N3, true, c * kTcRows}, Opnd{Zs, H, true, 0}, kTcRows, H,
                       false);
            mma_commit(&mbar);
        }
        if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
        phase ^= 1u;
        after_sync();
        // dZ2 = dR2 where R2 > 0, over R2 in Z; its column sums into db2
        for (int c = c0h; c < c1h; c += 8) {
            float v[8];
            tmem_ld8(tb + (uint32_t)c, v);
            uint4 *p = reinterpret_cast<uint4 *>(Zs + cm_off(row, c, H));
            const uint4 r2 = *p;
            const uint32_t rw[4] = {r2.x, r2.y, r2.z, r2.w};
            uint32_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float a = (rw[u] & 0x7FFFu) && live ? v[2 * u] : 0.f;
                const float b = (rw[u] & 0x7FFF0000u) && live ? v[2 * u + 1] : 0.f;
                v[2 * u] = a;
                v[2 * u + 1] = b;
                wv[u] = pack_bf16(a, b);
            }
            *p = make_uint4(wv[0], wv[1], wv[2], wv[3]);
#pragma unroll
            for (int u = 0; u < 8; ++u) col_sum_add(v[u], &db2[c + u]);
        }
        // dW3 rows of this lane (output n = 128 c + row), this half's columns, into the partial row
        for (int c = 0; c < nc; ++c) {
            const int nrow = c * kTcRows + row;
            const int j = nrow / SW, k = nrow - j * SW;
            for (int cc = c0h; cc < c1h; cc += 8) {
                float v[8];
                tmem_ld8(tb + 256u + (uint32_t)(c * H + cc), v);
                if (nrow < M3 && k < NO) add8(prow + pW3 + (j * NO + k) * H + cc, v, first);
            }
        }
        // ---- dR1 = dZ2 W2 into [0, H); dW2 = dZ2^T R1 into [H, 2H)
        to_mma();
        if (tid == 0) {
            mma_ab(tmem, Opnd{Zs, H, false, 0}, Opnd{W2, H, true, 0}, H, H, false);
            mma_ab(tmem + H, Opnd{Zs, H, true, 0}, Opnd{Ys, H, true, 0}, kTcRows, H, false);
            mma_commit(&mbar);
        }
        if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
        phase ^= 1u;
        after_sync();
        // dZ1 = dR1 where R1 > 0, over R1 in Y; its column sums into db1
        for (int c = c0h; c < c1h; c += 8) {
            float v[8];
            tmem_ld8(tb + (uint32_t)c, v);
            uint4 *p = reinterpret_cast<uint4 *>(Ys + cm_off(row, c, H));
            const uint4 r1 = *p;
            const uint32_t rw[4] = {r1.x, r1.y, r1.z, r1.w};
            uint32_t wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float a = (rw[u] & 0x7FFFu) && live ? v[2 * u] : 0.f;
                const float b = (rw[u] & 0x7FFF0000u) && live ? v[2 * u + 1] : 0.f;
                v[2 * u] = a;
                v[2 * u + 1] = b;
                wv[u] = pack_bf16(a, b);
            }
            *p = make_uint4(wv[0], wv[1], wv[2], wv[3]);
#pragma unroll
            for (int u = 0; u < 8; ++u) col_sum_add(v[u], &db1[c + u]);
        }
        // dW2 rows of this lane (output o = row < H)
        for (int cc = c0h; cc < c1h; cc += 8) {
            float v[8];
            tmem_ld8(tb + (uint32_t)(H + cc), v);
            if (row < H) add8(prow + pW2 + row * H + cc, v, first);
        }
        // ---- dA = dZ1 W1 into [0, 16); dW1 = dZ1^T A1 into [H, H + 16)
        to_mma();
        if (tid == 0) {
            mma_ab(tmem, Opnd{Ys, H, false, 0}, Opnd{W1, 16, true, 0}, H, 16, false);
            mma_ab(tmem + H, Opnd{Ys, H, true, 0}, Opnd{A1, 16, true, 0}, kTcRows, 16, false);
            mma_commit(&mbar);
        }
        if (!all_ok(mbar_wait(&mbar, phase))) { ok = false; break; }
        phase ^= 1u;
        after_sync();
        {
            float v[8];
            tmem_ld8(tb + (uint32_t)(8 * half), v);   // dA columns [8 half, 8 half + 8)
            if (live)
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int c = 8 * half + u;
                    if (c < nA) gin[sr * d + Y.A[c]] = gyA[u] + v[u];
                }
            tmem_ld8(tb + (uint32_t)(H + 8 * half), v);   // dW1 row h = row, columns [8 half, 8 half + 8)
            if (row < H)
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int c = 8 * half + u;
                    if (c < nA) {
                        float *dst = prow + row * nA + c;
                        *dst = first ? v[u] : *dst + v[u];
                    }
                }
        }
        before_sync();
        __syncthreads();   // the slabs and TMEM are reused by the next tile
        after_sync();
    }
    if (ok) {
        for (int o = tid; o < M3; o += kTT) {
            const int j = o / SW, k = o - j * SW;
            if (k < NO) prow[pb3 + j * NO + k] = db3[o];
        }
        for (int h = tid; h < H; h += kTT) {
            prow[pb2 + h] = db2[h];
            prow[pb1 + h] = db1[h];
        }
    }
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        if (copying) mbar_wait(&wbar, 0);   // the weight copy still writes this CTA's shared memory
    }
    before_sync();
    __syncthreads();
    after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBwdCols));
}

// ------------------------------------------------------------------------------ host
struct TcDev {
    int optin = 0, sms = 0;
};

int tc_dev(TcDev &out)
{
    static TcDev cache[64];
    static std::atomic<uint64_t> known{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev >= 0 && dev < 64 && (known.load(std::memory_order_acquire) >> dev & 1u)) {
        out = cache[dev];
        return MCUBES_OK;
    }
    TcDev t;
    e = cudaDeviceGetAttribute(&t.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&t.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev >= 0 && dev < 64) {
        cache[dev] = t;
        known.fetch_or(1ull << dev, std::memory_order_release);
    }
    out = t;
    return MCUBES_OK;
}

template <typename Kern>
int raise_limit(Kern kern, int optin, std::atomic<uint64_t> &done, int &avail)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return cuda_status(e);
    avail = optin - (int)fa.sharedSizeBytes;   // the opt-in limit covers static and dynamic shared memory
    if (dev >= 0 && dev < 64 && (done.load(std::memory_order_acquire) >> dev & 1u)) return MCUBES_OK;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, avail)) != cudaSuccess)
        return cuda_status(e);
    if (dev >= 0 && dev < 64) done.fetch_or(1ull << dev, std::memory_order_release);
    return MCUBES_OK;
}

template <int H, int K>
int tc_grad_hk(const TcFlow &F, const unsigned char *mirror, long long n, int d, const float *x, const float *w,
               int kind, float *grad, float *loss, const FusedTrainWork &W, cudaStream_t s)
{
    static std::atomic<uint64_t> fwd_done{0}, bwd_done{0};
    TcDev di;
    int st = tc_dev(di);
    if (st) return st;
    int fav = 0, bav = 0;
    if ((st = raise_limit(train_fwd_tc_kernel<H, K>, di.optin, fwd_done, fav))) return st;
    if ((st = raise_limit(train_bwd_tc_kernel<H, K>, di.optin, bwd_done, bav))) return st;
    const size_t wstride = (size_t)((F.max_bytes + 1023u) & ~1023u);
    const size_t rest = (size_t)kTcRows * 16 * 2 + (size_t)kTcRows * H * 2 + sizeof(float) * (size_t)kTcRows * (d | 1);
    int nbuf = 2;
    size_t fsm = 2 * wstride + rest;
    if (fsm > (size_t)fav) {
        nbuf = 1;
        fsm = wstride + rest;
    }
    const BwdTcSmem B = bwd_tc_smem<H>(F, d);
    if (fsm > (size_t)fav || B.total > (size_t)bav) return kFusedUnsupported;
    if ((st = cuda_status(cudaMemsetAsync(W.err, 0, sizeof(int), s)))) return st;
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    const unsigned fgrid = (unsigned)std::min<long long>(tiles, di.sms);
    train_fwd_tc_kernel<H, K><<<fgrid, kTT, fsm, s>>>(F, mirror, x, w, kind, d, n, W.hs, W.gl, loss, W.err, nbuf);
    if ((st = cuda_status(cudaGetLastError()))) return st;
    const int bgrid = (int)std::min<long long>(tiles, std::min<long long>(di.sms, W.part_rows));
    float *gout = nullptr, *gin = W.gA;
    for (int l = F.L - 1; l >= 0; --l) {
        const TcLayer &Y = F.lay[l];
        const int npl = (int)(Y.pb3 - Y.pW1) + Y.nB * (2 * K + 1);
        train_bwd_tc_kernel<H, K><<<(unsigned)bgrid, kTT, B.total, s>>>(
            F, mirror, l, B, W.hs + (size_t)l * (size_t)n * d, gout, W.gl, gin, d, n, W.part, W.part_stride, W.err);
        if ((st = cuda_status(cudaGetLastError()))) return st;
        if ((st = launch_reduce_part(W.part, bgrid, W.part_stride, npl, grad + Y.pW1, s))) return st;
        gout = gin;
        gin = (gin == W.gA) ? W.gB : W.gA;
    }
    return MCUBES_OK;
}

template <int H>
int tc_grad_h(const TcFlow &F, const unsigned char *mirror, long long n, int d, const float *x, const float *w,
              int kind, float *grad, float *loss, const FusedTrainWork &W, cudaStream_t s)
{
    switch (F.K) {
    case 4: return tc_grad_hk<H, 4>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    case 8: return tc_grad_hk<H, 8>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    case 16: return tc_grad_hk<H, 16>(F, mirror, n, d, x, w, kind, grad, loss, W, s);
    default: return kFusedUnsupported;
    }
}

}  // namespace

int tc_grad(const Shape &S, const float *params, long long n, const float *x, const float *w, int kind, float *grad,
            float *loss, const FusedTrainWork &W, size_t mirror_bytes, cudaStream_t s)
{
    if (n <= 0) return MCUBES_OK;
    if ((S.H != 64 && S.H != 128) || W.err == nullptr) return kFusedUnsupported;
    TcFlow F;
    if (!tc_layout(S, F) || F.total_bytes > mirror_bytes) return kFusedUnsupported;
    int st = build_tc_mirror(F, params, W.mirror, s);
    if (st) return st;
    switch (S.H) {
    case 64: return tc_grad_h<64>(F, W.mirror, n, S.d, x, w, kind, grad, loss, W, s);
    default: return tc_grad_h<128>(F, W.mirror, n, S.d, x, w, kind, grad, loss, W, s);
    }
}

}  // namespace flow
}  // namespace mcubes
