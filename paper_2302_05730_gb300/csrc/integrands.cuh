// Benchmark integrands of the m-Cubes V-Sample kernel: the Genz families behind the paper's
// f1..f6 (Sec. 5, Eq. 1-6), the addition integrand (Sec. 5.3) and a constant.
//
// The sampler produces the point one coordinate at a time, so each family is written as a
// running state fed coordinate by coordinate (add) and closed once per sample (finish).
//
// FP64 forms evaluate the family exactly as defined (params a = IntegrandParams::a, u = ::u).
//
// FP32 forms (the FP32-eval variant) return f / F, where F is a per-integrand FP64 factor
// the host folds back in (fscale). The host pre-scales the parameters:
//   oscillatory    fa = a / (2 pi), fc = u_0 mod 1; f/F = cos(2 pi (fc + sum fa x)); F = 1
//   product peak   fa = a, fu = u; f/F = 1 / prod(1 + (a (x - u))^2); F = prod a^2
//   corner peak    fa = a; f/F = (1 + sum a x)^-(d+1); F = 1
//   Gaussian       fa = a sqrt(log2 e), fu = u; f/F = 2^-(sum (fa (x - u))^2); F = 1
//   C0             fa = a log2 e, fu = u; f/F = 2^-(sum fa |x - u|); F = 1
//   discontinuous  fa = a log2 e, fu = u (the cut, rounded to single), fb = min(u, 1);
//                  f/F = 2^(sum fa (x - fb)) inside the cut, else 0; F = exp(sum a min(u,1))
//   addition       f/F = sum x; F = 1
//   constant       f/F = 1; F = a_0
//   double Gaussian fa = a sqrt(log2 e), fu = u, fb = 1 - u; f/F = 2^-s1 + 2^-s2; F = 1
//   rotated Gaussian fm = log2(e) M, fu = c; f/F = 2^-((x-c)^T fm (x-c)); F = 1
#pragma once

#include "common.cuh"

namespace mcubes {

enum : int {
    kOscillatory = 0,
    kProductPeak = 1,
    kCornerPeak = 2,
    kGaussian = 3,
    kC0 = 4,
    kDiscontinuous = 5,
    kAddition = 6,
    kConstant = 7,
    kDoubleGaussian = 8,
    kRotatedGaussian = 9,
    kNumIntegrands = 10
};

// 2^x, hardware approximation (relative error about 2^-22), subnormal results kept.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// base^(-e) for a compile-time e >= 1 by binary powering, then one reciprocal.
template <int E, typename T>
__device__ __forceinline__ T inv_pow(T base)
{
    T result = T(1);
    T b = base;
    int e = E;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        if (e & 1) result *= b;
        e >>= 1;
        if (e) b *= b;
    }
    return T(1) / result;
}

// ------------------------------------------------------------------------------ FP64 forms
template <int FID, int D>
struct Integrand64 {
    double s = 0.0;
    double s2 = 0.0;
    double prod = 1.0;
    bool inside = true;
    double xs[FID == kRotatedGaussian ? D : 1];

    __device__ __forceinline__ void add(int i, double x, const IntegrandParams &ip)
    {
        if constexpr (FID == kOscillatory || FID == kCornerPeak) {
            s = fma(ip.a[i], x, s);
        } else if constexpr (FID == kProductPeak) {
            const double t = x - ip.u[i];
            prod *= fma(t, t, ip.b[i]);                 // b = 1 / a^2
        } else if constexpr (FID == kGaussian) {
            const double v = ip.a[i] * (x - ip.u[i]);
            s = fma(v, v, s);
        } else if constexpr (FID == kC0) {
            s = fma(ip.a[i], fabs(x - ip.u[i]), s);
        } else if constexpr (FID == kDiscontinuous) {
            inside = inside && (x < ip.u[i]);
            s = fma(ip.a[i], x, s);
        } else if constexpr (FID == kAddition) {
            s += x;
        } else if constexpr (FID == kDoubleGaussian) {
            const double v1 = ip.a[i] * (x - ip.u[i]);
            const double v2 = ip.a[i] * (x - ip.b[i]);   // b = 1 - u
            s = fma(v1, v1, s);
            s2 = fma(v2, v2, s2);
        } else if constexpr (FID == kRotatedGaussian) {
            xs[i] = x - ip.u[i];
        }
    }

    __device__ __forceinline__ double finish(const IntegrandParams &ip) const
    {
        if constexpr (FID == kOscillatory) {
            return cos(fma(6.283185307179586476925286766559, ip.u[0], s));
        } else if constexpr (FID == kProductPeak) {
            return 1.0 / prod;
        } else if constexpr (FID == kCornerPeak) {
            return inv_pow<D + 1>(1.0 + s);
        } else if constexpr (FID == kGaussian || FID == kC0) {
            return exp(-s);
        } else if constexpr (FID == kDiscontinuous) {
            return inside ? exp(s) : 0.0;
        } else if constexpr (FID == kAddition) {
            return s;
        } else if constexpr (FID == kDoubleGaussian) {
            return exp(-s) + exp(-s2);
        } else if constexpr (FID == kRotatedGaussian) {
            double q = 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                double r = 0.0;
#pragma unroll
                for (int j = 0; j < D; ++j) r = fma(ip.m[i * D + j], xs[j], r);
                q = fma(xs[i], r, q);
            }
            return exp(-q);
        } else {
            return ip.a[0];
        }
    }
};

// ------------------------------------------------------------------------------ FP32 forms
template <int FID, int D>
struct Integrand32 {
    float s = 0.0f;
    float s2 = 0.0f;
    float prod = 1.0f;
    bool inside = true;
    float xs[FID == kRotatedGaussian ? D : 1];

    __device__ __forceinline__ void add(int i, float x, const IntegrandParams &ip)
    {
        if constexpr (FID == kOscillatory || FID == kCornerPeak) {
            s = fmaf(ip.fa[i], x, s);
        } else if constexpr (FID == kProductPeak) {
            const float v = ip.fa[i] * (x - ip.fu[i]);
            prod *= fmaf(v, v, 1.0f);
        } else if constexpr (FID == kGaussian) {
            const float v = ip.fa[i] * (x - ip.fu[i]);
            s = fmaf(v, v, s);
        } else if constexpr (FID == kC0) {
            s = fmaf(ip.fa[i], fabsf(x - ip.fu[i]), s);
        } else if constexpr (FID == kDiscontinuous) {
            inside = inside && (x < ip.fu[i]);
            s = fmaf(ip.fa[i], x - ip.fb[i], s);
        } else if constexpr (FID == kAddition) {
            s += x;
        } else if constexpr (FID == kDoubleGaussian) {
            const float v1 = ip.fa[i] * (x - ip.fu[i]);
            const float v2 = ip.fa[i] * (x - ip.fb[i]);
            s = fmaf(v1, v1, s);
            s2 = fmaf(v2, v2, s2);
        } else if constexpr (FID == kRotatedGaussian) {
            xs[i] = x - ip.fu[i];
        }
    }

    __device__ __forceinline__ float finish(const IntegrandParams &ip) const
    {
        if constexpr (FID == kOscillatory) {
            const float t = ip.fc + s;                  // phase in turns
            const float tr = t - rintf(t);              // [-1/2, 1/2]
            return __cosf(6.28318530717958647692f * tr);
        } else if constexpr (FID == kProductPeak) {
            return __frcp_rn(prod);
        } else if constexpr (FID == kCornerPeak) {
            return inv_pow<D + 1>(1.0f + s);
        } else if constexpr (FID == kGaussian || FID == kC0) {
            return ex2_approx(-s);
        } else if constexpr (FID == kDiscontinuous) {
            return inside ? ex2_approx(s) : 0.0f;
        } else if constexpr (FID == kAddition) {
            return s;
        } else if constexpr (FID == kDoubleGaussian) {
            return ex2_approx(-s) + ex2_approx(-s2);
        } else if constexpr (FID == kRotatedGaussian) {
            float q = 0.0f;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                float r = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) r = fmaf(ip.fm[i * D + j], xs[j], r);
                q = fmaf(xs[i], r, q);
            }
            return ex2_approx(-q);
        } else {
            return 1.0f;
        }
    }
};

}  // namespace mcubes
