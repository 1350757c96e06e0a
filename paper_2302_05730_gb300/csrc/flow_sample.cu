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
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mcubes.h"
#include "internal.h"
#include "integrands.cuh"

using namespace mcubes;

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

// FP32-layout uniform of axis i for sample (t, q): Philox call i / 4, word i % 4, low 23 bits.
__device__ __forceinline__ float uniform32(uint32_t t, uint32_t q, uint32_t ctr2_hi, uint32_t job, uint32_t k0,
                                           uint32_t k1, int i)
{
    const Words4 r = philox4x32_10(t, q, ctr2_hi | (uint32_t)(i >> 2), job, k0, k1);
    const uint32_t w = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
    return (float)(w & 0x7FFFFFu) * 1.1920928955078125e-7f;   // 2^-23
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
        for (int a = 0; a < S.d; ++a) {
            const float u = uniform32(t, q, S.ctr2_hi, S.job, S.key0, S.key1, a);
            float yn = ((float)c[a] + u) * R;
            yn = fminf(yn, 499.999969f);
            const int k = min((int)yn, kNB - 1);
            const double b0 = grid[a * kGS + k], b1 = grid[a * kGS + k + 1];
            const float wd = (float)(b1 - b0);
            xs[a] = fmaf(wd, yn - (float)k, (float)b0);
            J *= (float)kNB * wd;
            x[i * S.d + a] = xs[a];
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
        for (int a = 0; a < S.d; ++a) {
            const float u = uniform32(t, q, S.ctr2_hi, S.job, S.key0, S.key1, a);
            z[j * S.d + a] = fminf(((float)c[a] + u) * ig, 0.99999994f);
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
    const size_t wbytes = mcubes_flow_work_bytes(&sh, nwork);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bytes = al(sizeof(double) * d * kGS) + 2 * al(sizeof(float) * ntr * d) + 3 * al(sizeof(float) * ntr) +
                         4 * al(sizeof(float) * npar) + al(sizeof(float) * 2) + al(sizeof(double) * (2 * (size_t)cfg->flow_iters + 2)) +
                         2 * al(sizeof(float) * nchunk * d) + al(sizeof(float) * nchunk) + al(wbytes);
    char *mem = nullptr;
    if ((st = cuda_status(cudaMalloc(&mem, bytes)))) return st;
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
    if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
    out->seconds_train = seconds_since(t0);

    // ---- 4. m-Cubes iterations with the flow as proposal
    t0 = std::chrono::steady_clock::now();
    if ((st = cuda_status(cudaMemsetAsync(d_sums, 0, sizeof(double) * 2 * cfg->flow_iters, s)))) return finish(st);
    for (int it = 0; it < cfg->flow_iters; ++it) {
        SampleSpec F{(uint32_t)m, (uint32_t)p, (uint32_t)g, (uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32),
                     (uint32_t)(itmax + 2 + it) << 16, 0x20000000u, d, integrand_id};
        for (long long c0 = 0; c0 < m; c0 += chunk_cubes) {
            const long long nc = std::min<long long>(chunk_cubes, m - c0);
            const long long ns = nc * p;
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
    if (params_out &&
        (st = cuda_status(cudaMemcpyAsync(params_out, d_par, sizeof(float) * npar, cudaMemcpyDeviceToHost, s))))
        return finish(st);
    if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
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
