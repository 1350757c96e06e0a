// The learned proposal in use: m-Cubes with the coupling flow standing in for the VEGAS grid.
//   1. VEGAS adapts its grid for a few iterations (the library's own V-Sample and Rebin).
//   2. Samples drawn through the adapted grid are exported with their weights f^2 J
//      (variance loss) or |f| J (KL loss): the data the flow trains on, a fresh set per epoch.
//   3. The flow trains on them with the library's own forward, backward and Adam kernels.
//   4. m-Cubes iterations sample with the flow: the sub-cube strata live in latent space,
//      z = (c + u) / g, and x = flow^-1(z) carries density q(x). Each sample weighs f(x) / q(x),
//      and the per-cube mean and variance and the combination are as for the grid.
// The VEGAS grid stays: it seeds the training data, and its frozen-grid iterations at the same
// sample budget are the reference for each flow estimate's variance.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mcubes.h"
#include "flow_common.cuh"
#include "integrands.cuh"
#include "internal.h"

using namespace mcubes;
using flow::FusedFlow;
using flow::FusedLayer;
using flow::kFThreads;
using flow::kFWarps;
using flow::kFusedUnsupported;

namespace {

constexpr int kGS = kNB + 1;

// Integrand f / F in single precision for a runtime dimension (the FP32-eval forms of
// integrands.cuh written with loops).
__device__ float eval32(int fid, int d, const IntegrandParams &ip, const float *x)
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

// Digits of sub-cube t in base g (axis 0 fastest).
__device__ __forceinline__ void digits(uint32_t t, uint32_t g, int d, uint32_t *c)
{
    for (int i = 0; i < d; ++i) {
        c[i] = t % g;
        t /= g;
    }
}


struct SampleSpec {
    uint32_t m, p, g, key0, key1, ctr2_hi, job;
    int d, fid;
};

// Samples through the grid (as V-Sample draws them, single precision): x (n x d) and the weight
// w = (f / F) J for sample i = t p + q.
__global__ void vegas_export_kernel(const SampleSpec S, const IntegrandParams ip, const double *__restrict__ grid,
                                    long long n, float *__restrict__ x, float *__restrict__ w)
{
    const float R = (float)kNB / (float)S.g;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(i / S.p), q = (uint32_t)(i % S.p);
        uint32_t c[kDMax];
        digits(t, S.g, S.d, c);
        float xs[kDMax];
        float J = 1.f;
        for (int j = 0; 4 * j < S.d; ++j) {   // one Philox call per four axes
            float u[4];
            uniforms_f32x4(t, q, S.ctr2_hi, S.job, S.key0, S.key1, j, u);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int a = 4 * j + h;
                if (a >= S.d) break;
                float yn = ((float)c[a] + u[h]) * R;
                yn = fminf(yn, 499.999969f);
                const int k = min((int)yn, kNB - 1);
                const double b0 = grid[a * kGS + k], b1 = grid[a * kGS + k + 1];
                const float wd = (float)(b1 - b0);
                xs[a] = fmaf(wd, yn - (float)k, (float)b0);
                J *= (float)kNB * wd;
                x[i * S.d + a] = xs[a];
            }
        }
        w[i] = eval32(S.fid, S.d, ip, xs) * J;
    }
}

// Latent points stratified like V-Sample: z = (c + u) / g per axis, sample i = t p + q.
__global__ void latent_kernel(const SampleSpec S, long long i0, long long n, float *__restrict__ z)
{
    const float ig = 1.0f / (float)S.g;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const long long i = i0 + j;
        const uint32_t t = (uint32_t)(i / S.p), q = (uint32_t)(i % S.p);
        uint32_t c[kDMax];
        digits(t, S.g, S.d, c);
        for (int jc = 0; 4 * jc < S.d; ++jc) {   // one Philox call per four axes
            float u[4];
            uniforms_f32x4(t, q, S.ctr2_hi, S.job, S.key0, S.key1, jc, u);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int a = 4 * jc + h;
                if (a >= S.d) break;
                z[j * S.d + a] = fminf(((float)c[a] + u[h]) * ig, 0.99999994f);
            }
        }
    }
}

// One thread per sub-cube: weights f(x)/q(x) of its p samples, the cube's mean and variance,
// compensated per-thread sums, block reduction, two FP64 atomics (scaled by F).
__global__ void flow_eval_kernel(const SampleSpec S, const IntegrandParams ip, double fscale, long long ncubes, const float *__restrict__ x, const float *__restrict__ logq,
                                 double *__restrict__ sums)
{
    float cI = 0.f, eI = 0.f, cV = 0.f, eV = 0.f;
    const float inv_p = 1.0f / (float)S.p;
    for (long long tc = blockIdx.x * (long long)blockDim.x + threadIdx.x; tc < ncubes;
         tc += (long long)gridDim.x * blockDim.x) {
        float w0 = 0.f, S1 = 0.f, S2 = 0.f;
        for (uint32_t q = 0; q < S.p; ++q) {
            const long long j = tc * S.p + q;
            const float w = eval32(S.fid, S.d, ip, x + j * S.d) * __expf(-logq[j]);
            if (q == 0) {
                w0 = w;
            } else {
                const float dv = w - w0;
                S1 += dv;
                S2 = fmaf(dv, dv, S2);
            }
        }
        const float mean = fmaf(S1, inv_p, w0);
        const float var = fmaxf(fmaf(-S1 * inv_p, S1, S2), 0.f);
        const float tI = cI + mean;
        eI += (fabsf(cI) >= fabsf(mean)) ? ((cI - tI) + mean) : ((mean - tI) + cI);
        cI = tI;
        const float tV = cV + var;
        eV += (cV >= var) ? ((cV - tV) + var) : ((var - tV) + cV);
        cV = tV;
    }
    double sI = (double)cI + (double)eI, sV = (double)cV + (double)eV;
    for (int o = 16; o > 0; o >>= 1) {
        sI += __shfl_xor_sync(0xffffffffu, sI, o);
        sV += __shfl_xor_sync(0xffffffffu, sV, o);
    }
    __shared__ double red[2][32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wp] = sI;
        red[1][wp] = sV;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) {
            a += red[0][k];
            b += red[1][k];
        }
        const double pp = (double)S.p;
        atomicAdd(&sums[0], a * fscale);
        atomicAdd(&sums[1], b * fscale * fscale / (pp * (pp - 1.0)));
    }
}

// ------------------------------------------------------------------------------ fused sampling
// One launch takes a range of samples from their Philox draws to their weights:
//   z = (c + u) / g  ->  x = flow^-1(z), log q(x)  ->  w = (f(x) / F) exp(-log q(x)).
// A block holds 512 samples in shared memory and runs them through the layers one after the
// other. Each layer's weights are copied once per block and tile from a bf16 mirror that
// already has the padded shared-memory layout (16-byte copies). The MLP of a layer runs on the
// tensor cores (mma.sync m16n8k16, bf16 operands, FP32 accumulation); the hidden activations
// stay in registers between its three GEMMs, since the accumulator layout of one GEMM is the
// operand layout of the next. The output of the last GEMM goes to a per-warp shared buffer, two
// axes at a time, and each lane then transforms one (sample, axis) pair with the same
// pq_transform as the per-layer kernels.
// The bf16 mirror of the FP32 parameters in the fused kernels' shared layout: W1 [H][kK0 + 8],
// W2 [H][H + 8], W3 [round16(|B| SW)][H + 8] (slot j at rows j SW .. j SW + 2K), zero padding;
// biases FP32.
// blockIdx.y is the layer.
__global__ void mirror_kernel(const FusedFlow F, const float *__restrict__ p, unsigned char *__restrict__ mirror)
{
    const FusedLayer &Y = F.lay[blockIdx.y];
    const int H = F.H, LD0 = flow::kK0 + 8, LDH = H + 8, no = 2 * F.K + 1;
    unsigned char *base = mirror + Y.off;
    __nv_bfloat16 *W1 = reinterpret_cast<__nv_bfloat16 *>(base);
    __nv_bfloat16 *W2 = reinterpret_cast<__nv_bfloat16 *>(base + Y.oW2);
    __nv_bfloat16 *W3 = reinterpret_cast<__nv_bfloat16 *>(base + Y.oW3);
    float *b1 = reinterpret_cast<float *>(base + Y.ob1);
    float *b2 = reinterpret_cast<float *>(base + Y.ob2);
    float *b3 = reinterpret_cast<float *>(base + Y.ob3);
    const int n1 = H * LD0, n2 = H * LDH, n3 = flow::round16(Y.nB * F.SW) * LDH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2 + n3 + 2 * H + Y.nB * F.SW;
         e += gridDim.x * blockDim.x) {
        if (e < n1) {
            const int r = e / LD0, c = e - r * LD0;
            W1[e] = __float2bfloat16_rn(c < Y.nA ? p[Y.pW1 + r * Y.nA + c] : 0.f);
        } else if (e < n1 + n2) {
            const int f = e - n1, r = f / LDH, c = f - r * LDH;
            W2[f] = __float2bfloat16_rn(c < H ? p[Y.pW2 + r * H + c] : 0.f);
        } else if (e < n1 + n2 + n3) {
            const int f = e - n1 - n2, r = f / LDH, c = f - r * LDH, j = r / F.SW, k = r - j * F.SW;
            W3[f] = __float2bfloat16_rn((c < H && k < no && j < Y.nB) ? p[Y.pW3 + (j * no + k) * H + c] : 0.f);
        } else if (e < n1 + n2 + n3 + H) {
            b1[e - n1 - n2 - n3] = p[Y.pb1 + e - n1 - n2 - n3];
        } else if (e < n1 + n2 + n3 + 2 * H) {
            b2[e - n1 - n2 - n3 - H] = p[Y.pb2 + e - n1 - n2 - n3 - H];
        } else {
            const int f = e - n1 - n2 - n3 - 2 * H, j = f / F.SW, k = f - j * F.SW;
            b3[f] = k < no ? p[Y.pb3 + j * no + k] : 0.f;
        }
    }
}

template <int H, int K>
constexpr int fused_min_blocks()
{
    return H <= 64 ? 2 : 1;
}

constexpr int kFSub = 4, kFRows = kFWarps * 16 * kFSub;   // 512 samples per block tile

template <int H, int K>
size_t fused_smem(const FusedFlow &F, int d)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7;
    const int HS = d | 1;
    return (size_t)F.max_bytes + sizeof(float) * ((size_t)kFRows * HS + kFRows + (size_t)kFWarps * 2 * 16 * (SW + 1));
}

// Samples [i0, i0 + n) of one iteration (sample i = t p + q, t the sub-cube): x (optional,
// n x d), log q (optional) and the weight w = (f / F) / q, all indexed from i0.
template <int H, int K>
__global__ void __launch_bounds__(kFThreads, fused_min_blocks<H, K>())
    flow_sample_kernel(const FusedFlow F, const unsigned char *__restrict__ mirror, const SampleSpec S,
                       const IntegrandParams ip, long long i0, long long n, float *__restrict__ x_out,
                       float *__restrict__ lq_out, float *__restrict__ w_out)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, OS = SW + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int d = S.d, HS = d | 1;
    unsigned char *wbuf = smem;
    float *hs = reinterpret_cast<float *>(smem + F.max_bytes);
    float *lqs = hs + kFRows * HS;
    float *obuf = lqs + kFRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, row = lane & 15, half = lane >> 4;
    float *ob = obuf + warp * 2 * 16 * OS;
    const float ig = 1.0f / (float)S.g;
    const long long ntiles = (n + kFRows - 1) / kFRows;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long j0 = tile * kFRows;      // first sample of the tile, relative to i0
        for (int r = threadIdx.x; r < kFRows; r += kFThreads) {
            float *hr = hs + r * HS;
            if (j0 + r < n) {
                const long long i = i0 + j0 + r;
                const uint32_t tc = (uint32_t)(i / S.p), q = (uint32_t)(i % S.p);
                uint32_t c[kDMax];
                digits(tc, S.g, d, c);
                for (int jc = 0; 4 * jc < d; ++jc) {   // one Philox call per four axes
                    float u[4];
                    uniforms_f32x4(tc, q, S.ctr2_hi, S.job, S.key0, S.key1, jc, u);
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int a = 4 * jc + h;
                        if (a >= d) break;
                        hr[a] = fminf(((float)c[a] + u[h]) * ig, 0.99999994f);
                    }
                }
            } else {
                for (int a = 0; a < d; ++a) hr[a] = 0.5f;
            }
            lqs[r] = 0.f;
        }
        for (int l = F.L - 1; l >= 0; --l) {
            const FusedLayer &Y = F.lay[l];
            __syncthreads();   // the previous layer is done with the weight buffer; hs is complete
            {
                const uint4 *src = reinterpret_cast<const uint4 *>(mirror + Y.off);
                uint4 *dst = reinterpret_cast<uint4 *>(wbuf);
                for (uint32_t e = threadIdx.x; e < Y.bytes / 16u; e += kFThreads) dst[e] = src[e];
            }
            __syncthreads();
            for (int sub = 0; sub < kFSub; ++sub) {
                const int R0 = (warp * kFSub + sub) * 16;
                const float lq = flow::layer_rows16<H, K>(Y, wbuf, hs, HS, R0, ob, 1);
                if (half == 0) lqs[R0 + row] += lq;
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < kFRows; r += kFThreads) {
            const long long jr = j0 + r;
            if (jr >= n) continue;
            float x[kDMax];
            for (int a = 0; a < d; ++a) x[a] = hs[r * HS + a];
            const float lq = lqs[r];
            w_out[jr] = eval32(S.fid, d, ip, x) * __expf(-lq);
            if (x_out)
                for (int a = 0; a < d; ++a) x_out[jr * d + a] = x[a];
            if (lq_out) lq_out[jr] = lq;
        }
        __syncthreads();   // the next tile overwrites hs and lqs
    }
}

// Per-cube mean and variance of the weights w of ncubes whole sub-cubes (p samples each, from
// the first), compensated per-thread sums, block reduction, two FP64 atomics (scaled by F).
__global__ void cube_stats_kernel(const SampleSpec S, double fscale, long long ncubes, const float *__restrict__ wv,
                                  double *__restrict__ sums)
{
    float cI = 0.f, eI = 0.f, cV = 0.f, eV = 0.f;
    const float inv_p = 1.0f / (float)S.p;
    for (long long tc = blockIdx.x * (long long)blockDim.x + threadIdx.x; tc < ncubes;
         tc += (long long)gridDim.x * blockDim.x) {
        float w0 = 0.f, S1 = 0.f, S2 = 0.f;
        for (uint32_t q = 0; q < S.p; ++q) {
            const float w = wv[tc * S.p + q];
            if (q == 0) {
                w0 = w;
            } else {
                const float dv = w - w0;
                S1 += dv;
                S2 = fmaf(dv, dv, S2);
            }
        }
        const float mean = fmaf(S1, inv_p, w0);
        const float var = fmaxf(fmaf(-S1 * inv_p, S1, S2), 0.f);
        const float tI = cI + mean;
        eI += (fabsf(cI) >= fabsf(mean)) ? ((cI - tI) + mean) : ((mean - tI) + cI);
        cI = tI;
        const float tV = cV + var;
        eV += (cV >= var) ? ((cV - tV) + var) : ((var - tV) + cV);
        cV = tV;
    }
    double sI = (double)cI + (double)eI, sV = (double)cV + (double)eV;
    for (int o = 16; o > 0; o >>= 1) {
        sI += __shfl_xor_sync(0xffffffffu, sI, o);
        sV += __shfl_xor_sync(0xffffffffu, sV, o);
    }
    __shared__ double red[2][32];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wp] = sI;
        red[1][wp] = sV;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) {
            a += red[0][k];
            b += red[1][k];
        }
        const double pp = (double)S.p;
        atomicAdd(&sums[0], a * fscale);
        atomicAdd(&sums[1], b * fscale * fscale / (pp * (pp - 1.0)));
    }
}

template <int H, int K>
int launch_fused_hk(const FusedFlow &F, const unsigned char *mirror, const SampleSpec &S, const IntegrandParams &ip,
                    long long i0, long long n, float *x, float *lq, float *w, cudaStream_t s)
{
    const size_t smem = fused_smem<H, K>(F, S.d);
    // per device: the opt-in limit raised once to the device maximum, the limits read once
    static int optin_c[64], sms_c[64];
    static std::atomic<uint64_t> known{0};
    int dev = 0, optin = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 64 && (known.load(std::memory_order_acquire) >> dev & 1u)) {
        optin = optin_c[dev];
        sms = sms_c[dev];
    } else {
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, flow_sample_kernel<H, K>);
        if (e == cudaSuccess) {
            optin -= (int)fa.sharedSizeBytes;   // the opt-in limit covers static and dynamic shared memory
            e = cudaFuncSetAttribute(flow_sample_kernel<H, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        }
        if (e != cudaSuccess) return cuda_status(e);
        if (dev < 64) {
            optin_c[dev] = optin;
            sms_c[dev] = sms;
            known.fetch_or(1ull << dev, std::memory_order_release);
        }
    }
    if (smem > (size_t)optin) return kFusedUnsupported;
    // resident blocks per SM: shared memory (228 KB an SM, 1 KB reserved a block), then the
    // launch bound
    per_sm = std::max(1, std::min(fused_min_blocks<H, K>(), (int)(233472 / (smem + 1024))));
    const long long tiles = (n + kFRows - 1) / kFRows;
    const long long grid = std::min<long long>(tiles, (long long)per_sm * sms);
    flow_sample_kernel<H, K><<<(unsigned)grid, kFThreads, smem, s>>>(F, mirror, S, ip, i0, n, x, lq, w);
    return cuda_status(cudaGetLastError());
}

template <int H>
int launch_fused_h(const FusedFlow &F, const unsigned char *mirror, const SampleSpec &S, const IntegrandParams &ip,
                   long long i0, long long n, float *x, float *lq, float *w, cudaStream_t s)
{
    switch (F.K) {
    case 4: return launch_fused_hk<H, 4>(F, mirror, S, ip, i0, n, x, lq, w, s);
    case 8: return launch_fused_hk<H, 8>(F, mirror, S, ip, i0, n, x, lq, w, s);
    case 16: return launch_fused_hk<H, 16>(F, mirror, S, ip, i0, n, x, lq, w, s);
    case 32: return launch_fused_hk<H, 32>(F, mirror, S, ip, i0, n, x, lq, w, s);
    default: return MCUBES_ERR_INVALID_ARG;
    }
}

int launch_fused(const FusedFlow &F, const unsigned char *mirror, const SampleSpec &S, const IntegrandParams &ip,
                 long long i0, long long n, float *x, float *lq, float *w, cudaStream_t s)
{
    if (n <= 0) return MCUBES_OK;
    switch (F.H) {
    case 32: return launch_fused_h<32>(F, mirror, S, ip, i0, n, x, lq, w, s);
    case 64: return launch_fused_h<64>(F, mirror, S, ip, i0, n, x, lq, w, s);
    case 128: return launch_fused_h<128>(F, mirror, S, ip, i0, n, x, lq, w, s);
    default: return MCUBES_ERR_INVALID_ARG;
    }
}

// Weights for training: variance loss w^2, KL |w|, normalised so a batch of `batch` sums to 1
// (total read on the device; a set whose total is not positive and finite trains on zero weights).
__global__ void train_weights_kernel(const float *__restrict__ w, long long n, int kind, const double *__restrict__ total,
                                     double scale, float *__restrict__ out)
{
    const double tot = *total;
    const double f = (tot > 0.0 && tot < INFINITY) ? scale / tot : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = kind == 0 ? (double)w[i] * (double)w[i] : fabs((double)w[i]);
        out[i] = (float)(v * f);
    }
}

__global__ void sum_kernel(const float *__restrict__ w, long long n, int kind, double *__restrict__ out)
{
    double local = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        local += kind == 0 ? (double)w[i] * (double)w[i] : fabs((double)w[i]);
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, local);
}

// Seeded initial parameters: W1, W2 ~ N(0, 2/fan_in) (Box-Muller on Philox), biases 0, output
// layer 0 (the flow starts as the identity).
void init_params(const mcubes_flow_shape &sh, uint64_t seed, std::vector<float> &p)
{
    const int d = sh.d, L = sh.layers, H = sh.hidden, K = sh.bins;
    p.clear();
    uint32_t ctr = 0;
    auto normal = [&]() {
        const Words4 r = philox4x32_10(ctr++, 0x51A7u, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u1 = ((double)(r.x >> 8) + 0.5) / 16777216.0, u2 = (double)(r.y >> 8) / 16777216.0;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int l = 0; l < L; ++l) {
        const int kind = l % 4;
        int nA = 0;
        for (int i = 0; i < d; ++i) {
            bool inA = kind == 0 ? i < d / 2 : kind == 1 ? i >= d / 2 : kind == 2 ? (i % 2 == 0) : (i % 2 == 1);
            nA += inA;
        }
        const int nB = d - nA, nout = nB * (2 * K + 1);
        for (int i = 0; i < H * nA; ++i) p.push_back((float)(normal() * std::sqrt(2.0 / nA)));
        for (int i = 0; i < H; ++i) p.push_back(0.f);
        for (int i = 0; i < H * H; ++i) p.push_back((float)(normal() * std::sqrt(2.0 / H)));
        for (int i = 0; i < H; ++i) p.push_back(0.f);
        for (int i = 0; i < nout * H; ++i) p.push_back(0.f);
        for (int i = 0; i < nout; ++i) p.push_back(0.f);
    }
}

double seconds_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

namespace mcubes {
namespace flow {

int build_mirror(const FusedFlow &F, const float *d_params, unsigned char *mirror, cudaStream_t s)
{
    mirror_kernel<<<dim3(64, (unsigned)F.L), 256, 0, s>>>(F, d_params, mirror);
    return cuda_status(cudaGetLastError());
}

}  // namespace flow
}  // namespace mcubes

namespace {

// Scratch of the fused samplers: the larger of the two weight mirrors, then the tcgen05
// sampler's wait-expiry flag (256 bytes).
size_t sample_scratch(const flow::Shape &S, bool &tc_ok, flow::TcFlow &T, FusedFlow &F)
{
    const bool f_ok = flow::fused_layout(S, F);
    tc_ok = flow::tc_layout(S, T);
    if (!f_ok) return 0;
    const size_t m = std::max<size_t>(F.total_bytes, tc_ok ? T.total_bytes : 0);
    return ((m + 255) & ~(size_t)255) + 256;
}

}  // namespace

extern "C" size_t mcubes_flow_sample_work_bytes(const mcubes_flow_shape *shape)
{
    if (!shape || mcubes_flow_param_count(shape) <= 0) return 0;
    FusedFlow F;
    flow::TcFlow T;
    bool tc_ok;
    return sample_scratch(flow::Shape{shape->d, shape->layers, shape->hidden, shape->bins}, tc_ok, T, F);
}

extern "C" int mcubes_flow_sample_dev(const mcubes_flow_shape *shape, const float *d_params, int integrand_id,
                                      const double *params, int64_t ncall, uint64_t seed, int iteration, uint32_t job,
                                      int64_t i0, int64_t n, float *d_x, float *d_logq, float *d_w, double *fscale_out,
                                      void *d_work, size_t work_bytes, void *stream)
{
    if (!shape || !d_params || !params || !d_w || n < 0 || i0 < 0 || iteration < 0 || iteration > 0xFFFF)
        return MCUBES_ERR_INVALID_ARG;
    if (mcubes_flow_param_count(shape) <= 0) return MCUBES_ERR_INVALID_ARG;
    const flow::Shape S{shape->d, shape->layers, shape->hidden, shape->bins};
    FusedFlow F;
    flow::TcFlow T;
    bool tc_ok;
    const size_t need = sample_scratch(S, tc_ok, T, F);
    if (!need) return MCUBES_ERR_INVALID_ARG;
    if (!d_work || work_bytes < need || ((uintptr_t)d_work & 255u)) return MCUBES_ERR_WORKSPACE;
    Problem pb;
    int st = prepare(integrand_id, params, S.d, ncall, seed, 0, 0, 0, MCUBES_FP32_EVAL, pb);
    if (st) return st;
    if (i0 + n > pb.m * pb.p) return MCUBES_ERR_INVALID_ARG;
    if (fscale_out) *fscale_out = pb.P.fscale;
    const SampleSpec SS{(uint32_t)pb.m, (uint32_t)pb.p, (uint32_t)pb.g, (uint32_t)seed, (uint32_t)(seed >> 32),
                        (uint32_t)iteration << 16, job, S.d, integrand_id};
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *mirror = (unsigned char *)d_work;
    int *err = (int *)((char *)d_work + need - 256);
    if (tc_ok) {   // the tcgen05 sampler where the shape fits it
        if ((st = cuda_status(cudaMemsetAsync(err, 0, sizeof(int), s)))) return st;
        if ((st = flow::build_tc_mirror(T, d_params, mirror, s))) return st;
        const flow::TcSample TS{SS.m, SS.p, SS.g, SS.key0, SS.key1, SS.ctr2_hi, SS.job, SS.d, SS.fid};
        st = flow::launch_flow_sample_tc(T, mirror, TS, pb.P.ip, i0, n, d_x, d_logq, d_w, err, s);
        if (st != kFusedUnsupported) return st;
    }
    if ((st = flow::build_mirror(F, d_params, mirror, s))) return st;
    st = launch_fused(F, mirror, SS, pb.P.ip, i0, n, d_x, d_logq, d_w, s);
    return st == kFusedUnsupported ? MCUBES_ERR_INVALID_ARG : st;
}

extern "C" int mcubes_flow_integrate(int integrand_id, const double *params, int d, const mcubes_flow_config *cfg,
                                     float *params_out, mcubes_flow_report *out)
{
    if (!cfg || !out || !params) return MCUBES_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    const mcubes_flow_shape sh = cfg->shape;
    if (sh.d != d) return MCUBES_ERR_INVALID_ARG;
    const int64_t npar = mcubes_flow_param_count(&sh);
    if (npar <= 0) return MCUBES_ERR_INVALID_ARG;
    if (cfg->vegas_iters < 1 || cfg->flow_iters < 1 || cfg->train_steps < 0 || cfg->batch < 64 ||
        cfg->train_samples < cfg->batch || (cfg->loss_kind != 0 && cfg->loss_kind != 1) || !(cfg->lr > 0.f) ||
        cfg->ncall < 2 || cfg->vegas_iters + cfg->flow_iters > 0xFFF0)
        return MCUBES_ERR_INVALID_ARG;

    // ---- 1. VEGAS: vegas_iters adjusting iterations, then flow_iters frozen ones (the reference)
    const int itmax = cfg->vegas_iters + cfg->flow_iters;
    std::vector<double> grid((size_t)d * kGS), iters(2 * (size_t)itmax);
    auto t0 = std::chrono::steady_clock::now();
    int st = mcubes_integrate_range(integrand_id, params, d, cfg->ncall, itmax, cfg->vegas_iters, 0, itmax, cfg->seed,
                                    MCUBES_FP32_EVAL, nullptr, 0.0, grid.data(), iters.data(), nullptr);
    if (st) return st;
    out->seconds_vegas = seconds_since(t0);
    if ((st = mcubes_combine(iters.data(), itmax, cfg->vegas_iters, &out->vegas))) return st;
    int64_t g, m, p;
    if ((st = mcubes_stratify(d, cfg->ncall, &g, &m, &p))) return st;
    out->vegas.samples_per_iter = m * p;
    {
        double v = 0.0;
        for (int it = cfg->vegas_iters; it < itmax; ++it) v += iters[2 * it + 1];
        out->vegas_var_per_sample = v / cfg->flow_iters * (double)(m * p);
    }

    // integrand in its FP32-eval form (scale F)
    Problem pb;
    if ((st = prepare(integrand_id, params, d, cfg->ncall, cfg->seed, 0, 0, 0, MCUBES_FP32_EVAL, pb))) return st;

    // ---- device buffers
    const long long ntr = cfg->train_samples;
    const long long chunk_cubes = std::max<long long>(1, (1LL << 20) / p);
    const long long nchunk = chunk_cubes * p;
    const long long nwork = std::max<long long>(cfg->batch, nchunk);
    FusedFlow FF;
    flow::TcFlow TF;
    bool tc_ok = false;
    const size_t sample_bytes = sample_scratch(flow::Shape{sh.d, sh.layers, sh.hidden, sh.bins}, tc_ok, TF, FF);
    const bool fused_ok = sample_bytes > 0;
    const size_t wbytes = mcubes_flow_work_bytes(&sh, nwork);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bytes = al(sizeof(double) * d * kGS) + 2 * al(sizeof(float) * ntr * d) + 3 * al(sizeof(float) * ntr) +
                         4 * al(sizeof(float) * npar) + al(sizeof(float) * 2) + al(sizeof(double) * (2 * (size_t)cfg->flow_iters + 2)) +
                         2 * al(sizeof(float) * nchunk * d) + al(sizeof(float) * nchunk) + al(wbytes) +
                         al(fused_ok ? sample_bytes : 256);
    char *mem = nullptr;
    if ((st = cuda_status(mc_malloc((void **)&mem, bytes)))) return st;
    char *q = mem;
    auto take = [&](size_t b) { char *r = q; q += al(b); return r; };
    double *d_grid = (double *)take(sizeof(double) * d * kGS);
    float *d_x = (float *)take(sizeof(float) * ntr * d);
    float *d_wraw = (float *)take(sizeof(float) * ntr);
    float *d_w = (float *)take(sizeof(float) * ntr);
    float *d_par = (float *)take(sizeof(float) * npar);
    float *d_grad = (float *)take(sizeof(float) * npar);
    float *d_m = (float *)take(sizeof(float) * npar);
    float *d_v = (float *)take(sizeof(float) * npar);
    float *d_loss = (float *)take(sizeof(float) * 2);
    double *d_sums = (double *)take(sizeof(double) * (2 * (size_t)cfg->flow_iters + 2));
    float *d_z = (float *)take(sizeof(float) * nchunk * d);
    float *d_xs = (float *)take(sizeof(float) * nchunk * d);
    float *d_lq = (float *)take(sizeof(float) * nchunk);
    void *d_work = take(wbytes);
    unsigned char *d_mirror = (unsigned char *)take(fused_ok ? sample_bytes : 256);
    int *d_err = (int *)(d_mirror + (fused_ok ? sample_bytes : 256) - 256);
    cudaStream_t s = nullptr;
    auto finish = [&](int code) {
        if (s) cudaStreamDestroy(s);
        cudaFree(mem);
        return code;
    };
    if ((st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)))) return finish(st);

    // ---- 2. training data through the adapted grid. Each pass over the set (an epoch) draws a fresh
    // one from another Philox stream (job word 0x40000000 | epoch): the weights f J are heavy-tailed
    // wherever the grid misses the integrand's shape, and a fixed set lets the flow fit its few
    // largest points rather than the integrand.
    t0 = std::chrono::steady_clock::now();
    SampleSpec E;
    {
        int64_t ge, me, pe;
        // strata of the export: as many sub-cubes as a 2-point split of train_samples allows
        if ((st = mcubes_stratify(d, ntr, &ge, &me, &pe))) return finish(st);
        E = SampleSpec{(uint32_t)me, (uint32_t)(ntr / me), (uint32_t)ge, (uint32_t)cfg->seed,
                       (uint32_t)(cfg->seed >> 32), (uint32_t)(itmax + 1) << 16, 0x40000000u, d, integrand_id};
    }
    const long long nexp = (long long)E.m * E.p;   // <= train_samples
    const int batch = cfg->batch;
    if ((st = cuda_status(cudaMemcpyAsync(d_grid, grid.data(), sizeof(double) * d * kGS, cudaMemcpyHostToDevice, s))))
        return finish(st);
    double *d_tot = d_sums + 2 * (size_t)cfg->flow_iters;
    auto draw_training_set = [&](uint32_t epoch) -> int {
        SampleSpec Ee = E;
        Ee.job = 0x40000000u | (epoch & 0x0FFFFFFFu);
        vegas_export_kernel<<<(unsigned)std::min<long long>((nexp + 255) / 256, 65535), 256, 0, s>>>(Ee, pb.P.ip, d_grid,
                                                                                                      nexp, d_x, d_wraw);
        int e = cuda_status(cudaGetLastError());
        if (e) return e;
        if ((e = cuda_status(cudaMemsetAsync(d_tot, 0, sizeof(double), s)))) return e;
        sum_kernel<<<512, 256, 0, s>>>(d_wraw, nexp, cfg->loss_kind, d_tot);
        train_weights_kernel<<<512, 256, 0, s>>>(d_wraw, nexp, cfg->loss_kind, d_tot, (double)nexp / (double)batch, d_w);
        return cuda_status(cudaGetLastError());
    };
    if ((st = draw_training_set(0))) return finish(st);
    {
        double tot = 0.0;
        if ((st = cuda_status(cudaMemcpyAsync(&tot, d_tot, sizeof(double), cudaMemcpyDeviceToHost, s)))) return finish(st);
        if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
        if (!(tot > 0.0) || !std::isfinite(tot)) return finish(MCUBES_ERR_NONFINITE);
    }

    // ---- 3. train
    std::vector<float> h_par;
    init_params(sh, cfg->seed ^ 0x9E3779B97F4A7C15ull, h_par);
    if ((st = cuda_status(cudaMemcpyAsync(d_par, h_par.data(), sizeof(float) * npar, cudaMemcpyHostToDevice, s))))
        return finish(st);
    if ((st = cuda_status(cudaMemsetAsync(d_m, 0, sizeof(float) * npar, s)))) return finish(st);
    if ((st = cuda_status(cudaMemsetAsync(d_v, 0, sizeof(float) * npar, s)))) return finish(st);
    const long long nbatches = std::max<long long>(1, nexp / batch);
    for (int step = 1; step <= cfg->train_steps; ++step) {
        const long long b0 = ((step - 1) % nbatches) * (long long)batch;
        if (step > 1 && b0 == 0 && (st = draw_training_set((uint32_t)((step - 1) / nbatches)))) return finish(st);
        if ((st = cuda_status(cudaMemsetAsync(d_grad, 0, sizeof(float) * npar, s)))) return finish(st);
        if ((st = cuda_status(cudaMemsetAsync(d_loss, 0, sizeof(float), s)))) return finish(st);
        if ((st = mcubes_flow_grad_dev(&sh, d_par, batch, d_x + b0 * d, d_w + b0, cfg->loss_kind, d_grad, d_loss, d_work,
                                       wbytes, s)))
            return finish(st);
        // cosine decay of the rate to a tenth over the run keeps late steps from undoing the fit
        const float frac = cfg->train_steps > 1 ? (float)(step - 1) / (float)(cfg->train_steps - 1) : 0.f;
        const float lr = cfg->lr * (0.1f + 0.9f * 0.5f * (1.0f + std::cos(3.14159265f * frac)));
        if ((st = mcubes_flow_adam_dev(npar, d_par, d_grad, d_m, d_v, step, lr, s))) return finish(st);
        if (step == 1 || step == cfg->train_steps) {
            float l = 0.f;
            if ((st = cuda_status(cudaMemcpyAsync(&l, d_loss, sizeof(float), cudaMemcpyDeviceToHost, s)))) return finish(st);
            if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
            if (step == 1) out->train_loss_first = l;
            out->train_loss_last = l;
        }
    }
    {   // the tcgen05 training kernels' error word: the workspace's last 256 bytes
        int h_terr = 0;
        const int *d_terr = (const int *)((const char *)d_work + mcubes_flow_work_bytes(&sh, batch) - 256);
        if ((st = cuda_status(cudaMemcpyAsync(&h_terr, d_terr, sizeof(int), cudaMemcpyDeviceToHost, s)))) return finish(st);
        if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
        if (h_terr) return finish(MCUBES_ERR_TIMEOUT);
    }
    out->seconds_train = seconds_since(t0);

    // ---- 4. m-Cubes iterations with the flow as proposal: the fused sampling kernel where the
    // shape fits it (shared memory, at most 16 layers), else the per-layer kernels
    t0 = std::chrono::steady_clock::now();
    if ((st = cuda_status(cudaMemsetAsync(d_sums, 0, sizeof(double) * 2 * cfg->flow_iters, s)))) return finish(st);
    bool fused = fused_ok, use_tc = fused_ok && tc_ok;
    if ((st = cuda_status(cudaMemsetAsync(d_err, 0, sizeof(int), s)))) return finish(st);
    if (use_tc && (st = flow::build_tc_mirror(TF, d_par, d_mirror, s))) return finish(st);
    if (fused && !use_tc && (st = flow::build_mirror(FF, d_par, d_mirror, s))) return finish(st);
    for (int it = 0; it < cfg->flow_iters; ++it) {
        SampleSpec F{(uint32_t)m, (uint32_t)p, (uint32_t)g, (uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32),
                     (uint32_t)(itmax + 2 + it) << 16, 0x20000000u, d, integrand_id};
        for (long long c0 = 0; c0 < m; c0 += chunk_cubes) {
            const long long nc = std::min<long long>(chunk_cubes, m - c0);
            const long long ns = nc * p;
            if (use_tc) {
                const flow::TcSample TS{F.m, F.p, F.g, F.key0, F.key1, F.ctr2_hi, F.job, F.d, F.fid};
                st = flow::launch_flow_sample_tc(TF, d_mirror, TS, pb.P.ip, c0 * p, ns, nullptr, nullptr, d_lq, d_err, s);
                if (st == kFusedUnsupported) {   // switch to the mma.sync sampler for the rest
                    use_tc = false;
                    if ((st = flow::build_mirror(FF, d_par, d_mirror, s))) return finish(st);
                } else {
                    if (st) return finish(st);
                    cube_stats_kernel<<<(unsigned)std::min<long long>((nc + 255) / 256, 65535), 256, 0, s>>>(
                        F, pb.P.fscale, nc, d_lq, d_sums + 2 * it);
                    if ((st = cuda_status(cudaGetLastError()))) return finish(st);
                    continue;
                }
            }
            if (fused) {
                st = launch_fused(FF, d_mirror, F, pb.P.ip, c0 * p, ns, nullptr, nullptr, d_lq, s);
                if (st == kFusedUnsupported) {
                    fused = false;
                } else {
                    if (st) return finish(st);
                    cube_stats_kernel<<<(unsigned)std::min<long long>((nc + 255) / 256, 65535), 256, 0, s>>>(
                        F, pb.P.fscale, nc, d_lq, d_sums + 2 * it);
                    if ((st = cuda_status(cudaGetLastError()))) return finish(st);
                    continue;
                }
            }
            latent_kernel<<<(unsigned)std::min<long long>((ns + 255) / 256, 65535), 256, 0, s>>>(F, c0 * p, ns, d_z);
            if ((st = cuda_status(cudaGetLastError()))) return finish(st);
            if ((st = mcubes_flow_inverse_dev(&sh, d_par, ns, d_z, d_xs, d_lq, d_work, wbytes, s))) return finish(st);
            flow_eval_kernel<<<(unsigned)std::min<long long>((nc + 255) / 256, 65535), 256, 0, s>>>(
                F, pb.P.ip, pb.P.fscale, nc, d_xs, d_lq, d_sums + 2 * it);
            if ((st = cuda_status(cudaGetLastError()))) return finish(st);
        }
    }
    std::vector<double> fs(2 * (size_t)cfg->flow_iters);
    if ((st = cuda_status(cudaMemcpyAsync(fs.data(), d_sums, sizeof(double) * fs.size(), cudaMemcpyDeviceToHost, s))))
        return finish(st);
    int h_err = 0;
    if ((st = cuda_status(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s)))) return finish(st);
    if (params_out &&
        (st = cuda_status(cudaMemcpyAsync(params_out, d_par, sizeof(float) * npar, cudaMemcpyDeviceToHost, s))))
        return finish(st);
    if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
    if (h_err) return finish(MCUBES_ERR_TIMEOUT);
    out->seconds_flow = seconds_since(t0);
    std::vector<double> fi(2 * (size_t)cfg->flow_iters);
    double vsum = 0.0;
    for (int it = 0; it < cfg->flow_iters; ++it) {
        fi[2 * it] = fs[2 * it] / (double)m;
        fi[2 * it + 1] = fs[2 * it + 1] / ((double)m * (double)m);
        if (!std::isfinite(fi[2 * it]) || !std::isfinite(fi[2 * it + 1])) return finish(MCUBES_ERR_NONFINITE);
        vsum += fi[2 * it + 1];
    }
    out->flow_var_per_sample = vsum / cfg->flow_iters * (double)(m * p);
    if ((st = mcubes_combine(fi.data(), cfg->flow_iters, 0, &out->flow))) return finish(st);
    out->flow.samples_per_iter = m * p;
    return finish(MCUBES_OK);
}
