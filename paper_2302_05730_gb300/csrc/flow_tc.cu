// Fused flow sampler on the fifth-generation tensor cores (tcgen05, TMEM accumulators).
//
// A 256-thread CTA takes 128 samples at a time: sample row r is TMEM lane r of the accumulators,
// served by threads r and r + 128. Per coupling layer (sampling direction):
//   1. each thread writes its row's kept coordinates (bf16) into the GEMM-1 operand in shared
//      memory; one thread issues tcgen05.mma D1 = A1 W1^T (M = 128, N = H, K = 16) and commits
//      to an mbarrier;
//   2. each thread reads its row of D1 from TMEM (tcgen05.ld), adds the bias, applies ReLU and
//      writes the bf16 row into the GEMM-2 operand; D2 = A2 W2^T (K = H); the same again into
//      D3 = A3 W3^T (N = |B| SW rounded up to 16, at most 256);
//   3. each thread reads its row's 2K+1 outputs of every transformed axis straight from TMEM and
//      runs the piecewise-quadratic inverse (pq_transform) on them.
// After the last layer each thread evaluates the integrand at its point. Operands are bf16 in the
// K-major, unswizzled core-matrix layout (8 rows x 16 bytes per core matrix; leading-dimension
// offset 128 bytes between core matrices along K, stride offset K/8 x 128 bytes between 8-row
// groups); the weights come from a mirror that already has this layout.
//
// A layer's weights reach shared memory by one bulk asynchronous copy (cp.async.bulk, completed on
// an mbarrier by transaction bytes). With two weight buffers (when they fit), the copy of the next
// layer in the CTA's sequence (or of the next tile's first layer) is issued at the start of a
// layer and runs while that layer computes. Every mbarrier wait is bounded: on expiry the kernel
// records an error, waits (bounded) for its copies still in flight, stops and frees its TMEM.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/mcubes.h"
#include "flow_common.cuh"
#include "tc_common.cuh"
#include "integrands.cuh"
#include "internal.h"

namespace mcubes {
namespace flow {

namespace {

using namespace tc;

__device__ __forceinline__ float eval32_rt(int fid, int d, const IntegrandParams &ip, const float *x);

}  // namespace

// ------------------------------------------------------------------------------ mirror
bool tc_layout(const Shape &S, TcFlow &F)
{
    if (S.L > kFMaxLayers || S.H > 128) return false;
    std::memset(&F, 0, sizeof(F));
    F.L = S.L;
    F.H = S.H;
    F.K = S.K;
    F.SW = (2 * S.K + 1 + 7) & ~7;
    long long pos = 0;
    uint32_t off = 0;
    for (int l = 0; l < S.L; ++l) {
        const LayerDesc D = describe(S, l, pos);
        TcLayer &Y = F.lay[l];
        Y.nA = D.nA;
        Y.nB = D.nB;
        for (int i = 0; i < kMaxAB; ++i) {
            Y.A[i] = D.A[i];
            Y.B[i] = D.B[i];
        }
        Y.N3 = round16(D.nB * F.SW);
        if (Y.N3 > kTcCols) return false;
        Y.pW1 = (uint32_t)D.offW1;
        Y.pb1 = (uint32_t)D.offb1;
        Y.pW2 = (uint32_t)D.offW2;
        Y.pb2 = (uint32_t)D.offb2;
        Y.pW3 = (uint32_t)D.offW3;
        Y.pb3 = (uint32_t)D.offb3;
        uint32_t b = 2u * S.H * 16u;                  // W1: H x 16
        Y.oW2 = b;
        b += 2u * S.H * S.H;                          // W2: H x H
        Y.oW3 = b;
        b += 2u * (uint32_t)Y.N3 * S.H;               // W3: N3 x H
        Y.ob1 = b;
        b += 4u * S.H;
        Y.ob2 = b;
        b += 4u * S.H;
        Y.ob3 = b;
        b += 4u * (uint32_t)Y.N3;
        b = (b + 15u) & ~15u;
        Y.bytes = b;
        Y.off = off;
        off += b;
        F.max_bytes = std::max(F.max_bytes, b);
    }
    F.total_bytes = off;
    return true;
}

namespace {

// The bf16 mirror in the tcgen05 operand layout (blockIdx.y = layer).
__global__ void tc_mirror_kernel(const TcFlow F, const float *__restrict__ p, unsigned char *__restrict__ mirror)
{
    const TcLayer &Y = F.lay[blockIdx.y];
    const int H = F.H, no = 2 * F.K + 1, SW = F.SW;
    unsigned char *base = mirror + Y.off;
    const int n1 = H * 16, n2 = H * H, n3 = Y.N3 * H;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2 + n3 + 2 * H + Y.N3; e += gridDim.x * blockDim.x) {
        if (e < n1) {
            const int r = e / 16, c = e % 16;
            *reinterpret_cast<__nv_bfloat16 *>(base + cm_off(r, c, 16)) =
                __float2bfloat16_rn(c < Y.nA ? p[Y.pW1 + r * Y.nA + c] : 0.f);
        } else if (e < n1 + n2) {
            const int f = e - n1, r = f / H, c = f % H;
            *reinterpret_cast<__nv_bfloat16 *>(base + Y.oW2 + cm_off(r, c, H)) = __float2bfloat16_rn(p[Y.pW2 + r * H + c]);
        } else if (e < n1 + n2 + n3) {
            const int f = e - n1 - n2, r = f / H, c = f % H, j = r / SW, k = r % SW;
            const float v = (j < Y.nB && k < no) ? p[Y.pW3 + (j * no + k) * H + c] : 0.f;
            *reinterpret_cast<__nv_bfloat16 *>(base + Y.oW3 + cm_off(r, c, H)) = __float2bfloat16_rn(v);
        } else if (e < n1 + n2 + n3 + H) {
            const int f = e - n1 - n2 - n3;
            reinterpret_cast<float *>(base + Y.ob1)[f] = p[Y.pb1 + f];
        } else if (e < n1 + n2 + n3 + 2 * H) {
            const int f = e - n1 - n2 - n3 - H;
            reinterpret_cast<float *>(base + Y.ob2)[f] = p[Y.pb2 + f];
        } else {
            const int f = e - n1 - n2 - n3 - 2 * H, j = f / SW, k = f % SW;
            reinterpret_cast<float *>(base + Y.ob3)[f] = (j < Y.nB && k < no) ? p[Y.pb3 + j * no + k] : 0.f;
        }
    }
}

// Bias + ReLU of this thread's TMEM row, columns [half n/2, (half+1) n/2) of [col, col + n), into
// the bf16 operand row of an [128 x n] K-major core-matrix matrix.
__device__ __forceinline__ void relu_half(uint32_t taddr, const float *bias, unsigned char *op, int row, int n, int half)
{
    for (int c0 = half * (n >> 1); c0 < (half + 1) * (n >> 1); c0 += 8) {
        float v[8];
        tmem_ld8(taddr + (uint32_t)c0, v);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            w[j] = pack_bf16(fmaxf(v[2 * j] + bias[c0 + 2 * j], 0.f), fmaxf(v[2 * j + 1] + bias[c0 + 2 * j + 1], 0.f));
        *reinterpret_cast<uint4 *>(op + cm_off(row, c0, n)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

}  // namespace

// Samples [i0, i0 + n) of one iteration: x (optional), log q (optional), w = (f / F) / q.
// 256 threads: thread t serves row t mod 128 (TMEM lane; warps w and w + 4 read the same lanes),
// and its half h = t / 128 takes columns [h H/2, (h+1) H/2) of the ReLU epilogues and every other
// transformed axis (j = h, h + 2, ...) of the coupling transforms.
constexpr int kTcThreads = 2 * kTcRows;

template <int H, int K>
__global__ void __launch_bounds__(kTcThreads, 1)
    flow_sample_tc_kernel(const TcFlow F, const unsigned char *__restrict__ mirror, const TcSample S,
                          const IntegrandParams ip, long long i0, long long n, float *__restrict__ x_out,
                          float *__restrict__ lq_out, float *__restrict__ w_out, int *__restrict__ err, const int nbuf)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_holder;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t wbar[2];   // weight buffers: the bulk copies' completion
    __shared__ float lq_half[kTcRows];
    const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kTcRows - 1), half = tid >> 7, d = S.d, HS = d | 1;
    const uint32_t wstride = (F.max_bytes + 1023u) & ~1023u;
    unsigned char *const wbuf0 = smem, *const wbuf1 = smem + wstride;   // nbuf buffers of F.max_bytes
    unsigned char *A1 = smem + (size_t)nbuf * wstride;           // 128 x 16 bf16
    unsigned char *A2 = A1 + kTcRows * 16 * 2;                    // 128 x H bf16 (also GEMM-3 operand)
    float *hs = reinterpret_cast<float *>(A2 + kTcRows * H * 2);  // 128 x HS
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
    const float ig = 1.0f / (float)S.g;
    const long long ntiles = (n + kTcRows - 1) / kTcRows;
    // the CTA's layer sequence: step s is layer L - 1 - s mod L of its (s / L)-th tile, with
    // weights in buffer s mod nbuf, that buffer's (s / nbuf)-th use
    const long long my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long n_steps = my_tiles * F.L;
    uint32_t issued0 = 0u, issued1 = 0u, used0 = 0u, used1 = 0u;   // thread 0: copies issued / waited
    auto issue = [&](long long st) {
        const int b = (int)(st % nbuf);
        const TcLayer &Z = F.lay[F.L - 1 - (int)(st % F.L)];
        proxy_fence();   // earlier generic reads of the buffer come before the async write
        bulk_copy_g2s(b ? wbuf1 : wbuf0, mirror + Z.off, Z.bytes, &wbar[b]);
        if (b) ++issued1; else ++issued0;
    };
    if (tid == 0 && n_steps > 0) issue(0);
    long long step = 0;

    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long jr = tile * kTcRows + row;   // this row's sample, relative to i0
        if (half == 0) {
            if (jr < n) {
                const long long i = i0 + jr;
                const uint32_t tc = (uint32_t)(i / S.p), q = (uint32_t)(i % S.p);
                uint32_t t = tc;
                for (int jc = 0; 4 * jc < d; ++jc) {   // one Philox call per four axes
                    float u[4];
                    uniforms_f32x4(tc, q, S.ctr2_hi, S.job, S.key0, S.key1, jc, u);
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        if (4 * jc + h >= d) break;
                        const uint32_t c = t % S.g;
                        t /= S.g;
                        hr[4 * jc + h] = fminf(((float)c + u[h]) * ig, 0.99999994f);
                    }
                }
            } else {
                for (int a = 0; a < d; ++a) hr[a] = 0.5f;
            }
        }
        float lq = 0.f;
        for (int l = F.L - 1; l >= 0 && ok; --l, ++step) {
            const TcLayer &Y = F.lay[l];
            // the previous layer's MMAs, TMEM reads, bias reads and coordinate updates are complete
            before_sync();
            __syncthreads();
            after_sync();
            // the next step's weights into the other buffer (with one buffer: this step's), then
            // wait for this step's
            const int b = (int)(step % nbuf);
            if (tid == 0) {
                if (nbuf == 2 && step + 1 < n_steps) issue(step + 1);
                if (nbuf == 1) issue(step);
            }
            if (!__syncthreads_and(mbar_wait(&wbar[b], (uint32_t)((step / nbuf) & 1)))) { ok = false; break; }
            if (tid == 0) {
                if (b) ++used1; else ++used0;
            }
            const unsigned char *wbuf = b ? wbuf1 : wbuf0;
            const unsigned char *W1 = wbuf, *W2 = wbuf + Y.oW2, *W3 = wbuf + Y.oW3;
            const float *b1 = reinterpret_cast<const float *>(wbuf + Y.ob1);
            const float *b2 = reinterpret_cast<const float *>(wbuf + Y.ob2);
            const float *b3 = reinterpret_cast<const float *>(wbuf + Y.ob3);
            {   // GEMM-1 operand: this row's kept coordinates, columns >= |A| zero (each half 8 columns)
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c0 = 8 * half + 2 * j, c1 = c0 + 1;
                    w[j] = pack_bf16(c0 < Y.nA ? hr[Y.A[c0]] : 0.f, c1 < Y.nA ? hr[Y.A[c1]] : 0.f);
                }
                *reinterpret_cast<uint4 *>(A1 + cm_off(row, 8 * half, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
            proxy_fence();
            before_sync();
            __syncthreads();
            after_sync();
            if (tid == 0) {
                mma_issue(tmem, A1, W1, 16, H);
                mma_commit(&mbar);
            }
            if (!__syncthreads_and(mbar_wait(&mbar, phase))) { ok = false; break; }
            phase ^= 1u;
            after_sync();
            relu_half(lane_base, b1, A2, row, H, half);            // D1 at columns [0, H)
            proxy_fence();
            before_sync();
            __syncthreads();
            after_sync();
            if (tid == 0) {
                mma_issue(tmem + H, A2, W2, H, H);                 // D2 at columns [H, 2H)
                mma_commit(&mbar);
            }
            if (!__syncthreads_and(mbar_wait(&mbar, phase))) { ok = false; break; }   // GEMM 2 has read A2
            phase ^= 1u;
            after_sync();
            relu_half(lane_base + H, b2, A2, row, H, half);        // GEMM-3 operand over the GEMM-2 operand
            proxy_fence();
            before_sync();
            __syncthreads();
            after_sync();
            if (tid == 0) {
                mma_issue(tmem, A2, W3, H, Y.N3);                  // D3 at columns [0, N3)
                mma_commit(&mbar);
            }
            if (!__syncthreads_and(mbar_wait(&mbar, phase))) { ok = false; break; }
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
                pq_transform<K>(raw, hr[Y.B[j]], 1, out, qv);
                hr[Y.B[j]] = out;
                lq += __logf(qv);
            }
        }
        if (!ok) break;
        if (half == 1) lq_half[row] = lq;
        __syncthreads();
        if (half == 0 && jr < n) {
            lq += lq_half[row];
            float x[kDMax];
            for (int a = 0; a < d; ++a) x[a] = hr[a];
            w_out[jr] = eval32_rt(S.fid, d, ip, x) * __expf(-lq);
            if (x_out)
                for (int a = 0; a < d; ++a) x_out[jr * d + a] = x[a];
            if (lq_out) lq_out[jr] = lq;
        }
    }
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        // bulk copies still in flight write this CTA's shared memory: wait for them (bounded)
        for (; used0 < issued0; ++used0) mbar_wait(&wbar[0], used0 & 1u);
        for (; used1 < issued1; ++used1) mbar_wait(&wbar[1], used1 & 1u);
    }
    before_sync();
    __syncthreads();
    after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

namespace {

// The integrand f / F in single precision for a runtime dimension (the FP32-eval forms).
__device__ __forceinline__ float eval32_rt(int fid, int d, const IntegrandParams &ip, const float *x)
{
    float s = 0.f, s2 = 0.f, prod = 1.f;
    bool inside = true;
    switch (fid) {
    case kOscillatory: {
        for (int i = 0; i < d; ++i) s = fmaf(ip.fa[i], x[i], s);
        const float t = ip.fc + s;
        return __cosf(6.28318530717958647692f * (t - rintf(t)));
    }
    case kProductPeak:
        for (int i = 0; i < d; ++i) {
            const float v = ip.fa[i] * (x[i] - ip.fu[i]);
            prod *= fmaf(v, v, 1.0f);
        }
        return __frcp_rn(prod);
    case kCornerPeak: {
        for (int i = 0; i < d; ++i) s = fmaf(ip.fa[i], x[i], s);
        const float b = 1.0f + s;
        float r = 1.0f;
        for (int e = 0; e <= d; ++e) r *= b;
        return 1.0f / r;
    }
    case kGaussian:
        for (int i = 0; i < d; ++i) {
            const float v = ip.fa[i] * (x[i] - ip.fu[i]);
            s = fmaf(v, v, s);
        }
        return ex2_approx(-s);
    case kC0:
        for (int i = 0; i < d; ++i) s = fmaf(ip.fa[i], fabsf(x[i] - ip.fu[i]), s);
        return ex2_approx(-s);
    case kDiscontinuous:
        for (int i = 0; i < d; ++i) {
            inside = inside && (x[i] < ip.fu[i]);
            s = fmaf(ip.fa[i], x[i] - ip.fb[i], s);
        }
        return inside ? ex2_approx(s) : 0.f;
    case kAddition:
        for (int i = 0; i < d; ++i) s += x[i];
        return s;
    case kDoubleGaussian:
        for (int i = 0; i < d; ++i) {
            const float v1 = ip.fa[i] * (x[i] - ip.fu[i]);
            const float v2 = ip.fa[i] * (x[i] - ip.fb[i]);
            s = fmaf(v1, v1, s);
            s2 = fmaf(v2, v2, s2);
        }
        return ex2_approx(-s) + ex2_approx(-s2);
    case kRotatedGaussian: {
        for (int i = 0; i < d; ++i) {
            float r = 0.f;
            for (int j = 0; j < d; ++j) r = fmaf(ip.fm[i * d + j], x[j] - ip.fu[j], r);
            s = fmaf(x[i] - ip.fu[i], r, s);
        }
        return ex2_approx(-s);
    }
    default:
        return 1.0f;
    }
}

template <int H, int K>
int launch_tc_hk(const TcFlow &F, const unsigned char *mirror, const TcSample &S, const IntegrandParams &ip,
                 long long i0, long long n, float *x, float *lq, float *w, int *err, cudaStream_t s)
{
    static int optin_c[64], sms_c[64];
    static std::atomic<uint64_t> known{0};
    int dev = 0, optin = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 64 && (known.load(std::memory_order_acquire) >> dev & 1u)) {
        optin = optin_c[dev];
        sms = sms_c[dev];
    } else {
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, flow_sample_tc_kernel<H, K>);
        if (e == cudaSuccess) {
            optin -= (int)fa.sharedSizeBytes;   // the opt-in limit covers static and dynamic shared memory
            e = cudaFuncSetAttribute(flow_sample_tc_kernel<H, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        }
        if (e != cudaSuccess) return cuda_status(e);
        if (dev < 64) {
            optin_c[dev] = optin;
            sms_c[dev] = sms;
            known.fetch_or(1ull << dev, std::memory_order_release);
        }
    }
    const int HS = S.d | 1;
    const size_t wstride = (size_t)((F.max_bytes + 1023u) & ~1023u);
    const size_t rest = (size_t)kTcRows * 16 * 2 + (size_t)kTcRows * H * 2 + sizeof(float) * (size_t)kTcRows * HS;
    // two weight buffers (the next layer's copy overlaps this layer) when two CTAs an SM still fit
    // them, else one
    int nbuf = 2;
    size_t smem = 2 * wstride + rest;
    if (2 * (smem + 1024) > (size_t)optin) {
        nbuf = 1;
        smem = wstride + rest;
    }
    // TMEM holds 512 columns an SM and a CTA takes kTcCols: a third resident CTA would wait in
    // tcgen05.alloc, so shared memory is padded to keep at most two on an SM
    smem = std::max(smem, (size_t)80 * 1024);
    if (smem + 1024 > (size_t)optin) return kFusedUnsupported;
    const int per_sm = 512 / kTcCols;
    const long long tiles = (n + kTcRows - 1) / kTcRows;
    const long long grid = std::min<long long>(tiles, (long long)per_sm * sms);
    flow_sample_tc_kernel<H, K><<<(unsigned)grid, kTcThreads, smem, s>>>(F, mirror, S, ip, i0, n, x, lq, w, err, nbuf);
    return cuda_status(cudaGetLastError());
}

template <int H>
int launch_tc_h(const TcFlow &F, const unsigned char *mirror, const TcSample &S, const IntegrandParams &ip,
                long long i0, long long n, float *x, float *lq, float *w, int *err, cudaStream_t s)
{
    switch (F.K) {
    case 4: return launch_tc_hk<H, 4>(F, mirror, S, ip, i0, n, x, lq, w, err, s);
    case 8: return launch_tc_hk<H, 8>(F, mirror, S, ip, i0, n, x, lq, w, err, s);
    case 16: return launch_tc_hk<H, 16>(F, mirror, S, ip, i0, n, x, lq, w, err, s);
    default: return kFusedUnsupported;   // K = 32: the raw row does not fit the registers well
    }
}

}  // namespace

int build_tc_mirror(const TcFlow &F, const float *d_params, unsigned char *mirror, cudaStream_t s)
{
    tc_mirror_kernel<<<dim3(64, (unsigned)F.L), 256, 0, s>>>(F, d_params, mirror);
    return cuda_status(cudaGetLastError());
}

int launch_flow_sample_tc(const TcFlow &F, const unsigned char *mirror, const TcSample &S, const IntegrandParams &ip,
                          long long i0, long long n, float *x, float *lq, float *w, int *err, cudaStream_t s)
{
    if (n <= 0) return MCUBES_OK;
    switch (F.H) {
    case 32: return launch_tc_h<32>(F, mirror, S, ip, i0, n, x, lq, w, err, s);
    case 64: return launch_tc_h<64>(F, mirror, S, ip, i0, n, x, lq, w, err, s);
    case 128: return launch_tc_h<128>(F, mirror, S, ip, i0, n, x, lq, w, err, s);
    default: return kFusedUnsupported;
    }
}

}  // namespace flow
}  // namespace mcubes
