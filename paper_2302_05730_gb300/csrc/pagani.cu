// PAGANI, the paper's other workload (Sec. 3.1): the region-evaluation kernel (the PAGANI-kernel
// algorithm) and an adaptive driver whose classify / split steps also run on the device.
//
// Evaluation. A warp takes one region (low corner lo, side lengths len) and its lanes stride over
// the f_eval points of a fully symmetric cubature rule on the region; each lane keeps the five
// class sums of its points in registers, the centre and the axis points go to shared memory for
// the split-axis test, the class sums are warp-reduced, and lane 0 forms the estimates. The rule
// (the paper defers it to PAGANI) is the published Genz-Malik rule of degree 7 with its embedded
// rule of degree 5 on the reference cube [-1, 1]^d:
//   classes 1: centre; 2: +-l2 e_i; 3: +-l3 e_i; 4: +-l4 e_i +- l4 e_j (i < j); 5: all (+-l5, ...),
//   l2^2 = 9/70, l3^2 = l4^2 = 9/10, l5^2 = 9/19, f_eval = 1 + 4d + 2d(d-1) + 2^d;
//   degree-7 weights 2^d (12824 - 9120 d + 400 d^2)/19683, 2^d 980/6561, 2^d (1820 - 400 d)/19683,
//   2^d 200/19683, 6859/19683; degree-5 weights 2^d (729 - 950 d + 50 d^2)/729, 2^d 245/486,
//   2^d (265 - 100 d)/1458, 2^d 25/729, 0.
// Five rules per region, as the paper's kernel accumulates: R7 and R5 above, and from the moment
// conditions (exact for 1 and x_i^2) R3a on classes 1, 2 (w2 = 2^d / (6 l2^2), w1 = 2^d - 2d w2),
// R3b on classes 1, 3 (w3 = 2^d / (6 l3^2), w1 = 2^d - 2d w3) and R1, the centre (w1 = 2^d).
// I = R7 (scaled by volume / 2^d). E from the differences of successive degrees, D7 = |R7 - R5|,
// D5 = max(|R5 - R3a|, |R5 - R3b|), D3 = max(|R3a - R1|, |R3b - R1|): E = D7 when D7 <= D5 / 4 and
// D5 <= D3 / 4 (the asymptotic range), else max(D7, D5, D3). Split axis = the largest fourth divided difference
// |f(l2 e_i) + f(-l2 e_i) - 2 f(0) - (l2/l3)^2 (f(l3 e_i) + f(-l3 e_i) - 2 f(0))|, ties to the
// longest side, then the lowest axis; differences within 1e-12 of the larger one and of the
// largest |f| at the centre and axis points tie (below that they are rounding noise). FP64
// throughout (the paper's precision).
//
// Adaptive driver (the paper describes the kernel only; this is the reading): the unit cube starts
// as init_split^d regions; every iteration evaluates the active regions, stops once the running
// E <= rel_tol |I|, finishes a region whose error is within its share of the budget
// (E_r <= rel_tol |I| V_r), and halves every other region along its split axis, children in the
// parents' order (an order-preserving scan).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mcubes.h"
#include "integrands.cuh"
#include "internal.h"

using namespace mcubes;

namespace {

constexpr int kPgWarps = 4;                     // regions per block
constexpr int kPgAxisPts = 1 + 4 * kDMax;       // centre + classes 2 and 3
constexpr int kScanBlock = 1024;

struct PgRule {
    int d, n, base3, base4, base5;
    double l2, l3, l4, l5, r23;
    double w[5][5];   // class weights of the rules R7, R5, R3a, R3b, R1
};

PgRule make_rule(int d)
{
    PgRule R;
    R.d = d;
    R.base3 = 1 + 2 * d;
    R.base4 = 1 + 4 * d;
    R.base5 = 1 + 4 * d + 2 * d * (d - 1);
    R.n = R.base5 + (1 << d);
    R.l2 = std::sqrt(9.0 / 70.0);
    R.l3 = std::sqrt(9.0 / 10.0);
    R.l4 = std::sqrt(9.0 / 10.0);
    R.l5 = std::sqrt(9.0 / 19.0);
    R.r23 = (9.0 / 70.0) / (9.0 / 10.0);
    const double p2 = std::ldexp(1.0, d), dd = (double)d;
    std::memset(R.w, 0, sizeof(R.w));
    R.w[0][0] = p2 * (12824.0 - 9120.0 * dd + 400.0 * dd * dd) / 19683.0;
    R.w[0][1] = p2 * 980.0 / 6561.0;
    R.w[0][2] = p2 * (1820.0 - 400.0 * dd) / 19683.0;
    R.w[0][3] = p2 * 200.0 / 19683.0;
    R.w[0][4] = 6859.0 / 19683.0;
    R.w[1][0] = p2 * (729.0 - 950.0 * dd + 50.0 * dd * dd) / 729.0;
    R.w[1][1] = p2 * 245.0 / 486.0;
    R.w[1][2] = p2 * (265.0 - 100.0 * dd) / 1458.0;
    R.w[1][3] = p2 * 25.0 / 729.0;
    R.w[2][1] = p2 / (6.0 * (9.0 / 70.0));
    R.w[2][0] = p2 - 2.0 * dd * R.w[2][1];
    R.w[3][2] = p2 / (6.0 * (9.0 / 10.0));
    R.w[3][0] = p2 - 2.0 * dd * R.w[3][2];
    R.w[4][0] = p2;
    return R;
}

// The integrand in FP64 for a runtime dimension (the FP64 forms of integrands.cuh written with loops).
__device__ double eval64(int fid, int d, const IntegrandParams &ip, const double *x)
{
    double s = 0.0, s2 = 0.0, prod = 1.0;
    bool inside = true;
    switch (fid) {
    case kOscillatory:
        for (int i = 0; i < d; ++i) s = fma(ip.a[i], x[i], s);
        return cos(fma(6.283185307179586476925286766559, ip.u[0], s));
    case kProductPeak:
        for (int i = 0; i < d; ++i) {
            const double t = x[i] - ip.u[i];
            prod *= fma(t, t, ip.b[i]);
        }
        return 1.0 / prod;
    case kCornerPeak: {
        for (int i = 0; i < d; ++i) s = fma(ip.a[i], x[i], s);
        const double b = 1.0 + s;
        double r = 1.0;
        for (int e = 0; e <= d; ++e) r *= b;
        return 1.0 / r;
    }
    case kGaussian:
        for (int i = 0; i < d; ++i) {
            const double v = ip.a[i] * (x[i] - ip.u[i]);
            s = fma(v, v, s);
        }
        return exp(-s);
    case kC0:
        for (int i = 0; i < d; ++i) s = fma(ip.a[i], fabs(x[i] - ip.u[i]), s);
        return exp(-s);
    case kDiscontinuous:
        for (int i = 0; i < d; ++i) {
            inside = inside && (x[i] < ip.u[i]);
            s = fma(ip.a[i], x[i], s);
        }
        return inside ? exp(s) : 0.0;
    case kAddition:
        for (int i = 0; i < d; ++i) s += x[i];
        return s;
    case kDoubleGaussian:
        for (int i = 0; i < d; ++i) {
            const double v1 = ip.a[i] * (x[i] - ip.u[i]);
            const double v2 = ip.a[i] * (x[i] - ip.b[i]);
            s = fma(v1, v1, s);
            s2 = fma(v2, v2, s2);
        }
        return exp(-s) + exp(-s2);
    case kRotatedGaussian: {
        double q = 0.0;
        for (int i = 0; i < d; ++i) {
            double r = 0.0;
            for (int j = 0; j < d; ++j) r = fma(ip.m[i * d + j], x[j] - ip.u[j], r);
            q = fma(x[i] - ip.u[i], r, q);
        }
        return exp(-q);
    }
    default:
        return ip.a[0];
    }
}

// A region's estimates from its class sums S and its centre and axis values fax: I = R7, E from
// the five rules (above) and the split axis (largest fourth difference; ties -- within 1e-12 of the
// larger difference and of the largest |f| at those points -- to the longest side, then the
// lowest axis).
__device__ void finish_region(const PgRule &R, const double (&S)[5], const double *fax, const double *rlen,
                              double *I, double *E, int *axis)
{
    const int d = R.d;
    double vol = 1.0;
    for (int i = 0; i < d; ++i) vol *= rlen[i];
    const double scale = vol / ldexp(1.0, d);
    double Q[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < 5; ++k) v += R.w[r][k] * S[k];
        Q[r] = v * scale;
    }
    *I = Q[0];
    const double d7 = fabs(Q[0] - Q[1]);
    const double d5 = fmax(fabs(Q[1] - Q[2]), fabs(Q[1] - Q[3]));
    const double d3 = fmax(fabs(Q[2] - Q[4]), fabs(Q[3] - Q[4]));
    *E = (d7 <= 0.25 * d5 && d5 <= 0.25 * d3) ? d7 : fmax(d7, fmax(d5, d3));
    const double f0 = fax[0];
    double fscale = fabs(f0);   // the rounding-noise scale of the fourth differences
    for (int p = 1; p < R.base4; ++p) fscale = fmax(fscale, fabs(fax[p]));
    double best = -1.0;
    int bi = 0;
    for (int i = 0; i < d; ++i) {
        const double a2 = fax[1 + 2 * i] + fax[2 + 2 * i] - 2.0 * f0;
        const double a3 = fax[R.base3 + 2 * i] + fax[R.base3 + 1 + 2 * i] - 2.0 * f0;
        const double D = fabs(a2 - R.r23 * a3);
        const double tie = 1e-12 * fmax(fmax(D, best), fscale);
        if (D > best + tie) {
            best = D;
            bi = i;
        } else if (fabs(D - best) <= tie && rlen[i] > rlen[bi]) {
            bi = i;
        }
    }
    *axis = bi;
}

// Rule point p on [-1, 1]^d (the oracle's order): u, and its class 1..5.
__device__ __forceinline__ int rule_point(const PgRule &R, int p, double *u)
{
    const int d = R.d;
    for (int i = 0; i < d; ++i) u[i] = 0.0;
    if (p == 0) return 1;
    if (p < R.base3) {
        const int q = p - 1;
        u[q >> 1] = (q & 1) ? -R.l2 : R.l2;
        return 2;
    }
    if (p < R.base4) {
        const int q = p - R.base3;
        u[q >> 1] = (q & 1) ? -R.l3 : R.l3;
        return 3;
    }
    if (p < R.base5) {
        const int q = p - R.base4, sg = q & 3;
        int pair = q >> 2, i = 0;
        while (pair >= d - 1 - i) {   // pairs i < j in row-major order
            pair -= d - 1 - i;
            ++i;
        }
        const int j = i + 1 + pair;
        u[i] = (sg & 2) ? -R.l4 : R.l4;
        u[j] = (sg & 1) ? -R.l4 : R.l4;
        return 4;
    }
    const int b = p - R.base5;
    for (int i = 0; i < d; ++i) u[i] = ((b >> i) & 1) ? -R.l5 : R.l5;
    return 5;
}

// Separable families. A rule point's coordinate on axis i takes one of 9 values (u = 0, +-l2, +-l3,
// +-l4, +-l5), so a warp tabulates each axis's factor or term at those 9 points once per region, and
// a point combines table entries instead of evaluating the integrand from scratch:
//   multiplicative (no transcendental per point): f = prod_i e_i(x_i) with e = exp(-phi) for the
//   Gaussian and C0, exp(a x) for the discontinuous family (times its cut), 1 / psi for the product
//   peak; the double Gaussian is the sum of two such products;
//   additive: f = g(sum_i phi_i(x_i)) for the oscillatory (cos), corner peak and addition families.
// Classes 1-4 change at most two axes from the centre: they use the centre's product over all but
// those axes (tabulated per axis and per pair), so no factor is divided out (a factor can underflow
// to zero). Class 5 combines d table entries.
constexpr int kPgMaxPairs = kDMax * (kDMax - 1) / 2;

struct PgAxisTab {
    double t1[kDMax][9];          // per-axis factor (multiplicative) or term (additive)
    double t2[kDMax][9];          // double Gaussian: the second peak's factors
    unsigned char out[kDMax][9];  // discontinuous: 1 where x_i >= u_i (outside the cut)
    double ex1[kDMax], ex2[kDMax];            // centre product (or sum) over all axes but k
    double px1[kPgMaxPairs], px2[kPgMaxPairs];   // ... over all axes but the pair (i, j)
    int nout_ex1[kDMax], nout_px[kPgMaxPairs];   // discontinuous: centre cut count without k / (i, j)
    double all1, all2;
    int nout_all;
};

__device__ __forceinline__ bool pg_mult(int fid)
{
    return fid == kGaussian || fid == kC0 || fid == kDiscontinuous || fid == kDoubleGaussian || fid == kProductPeak;
}

// The factor / term of axis i at coordinate x.
__device__ __forceinline__ void pg_terms(int fid, const IntegrandParams &ip, int i, double x, double &t1, double &t2,
                                         unsigned char &out)
{
    t2 = 0.0;
    out = 0;
    switch (fid) {
    case kOscillatory:
    case kCornerPeak:
        t1 = ip.a[i] * x;
        break;
    case kProductPeak: {
        const double t = x - ip.u[i];
        t1 = 1.0 / fma(t, t, ip.b[i]);
        break;
    }
    case kGaussian: {
        const double v = ip.a[i] * (x - ip.u[i]);
        t1 = exp(-(v * v));
        break;
    }
    case kC0:
        t1 = exp(-(ip.a[i] * fabs(x - ip.u[i])));
        break;
    case kDiscontinuous:
        t1 = exp(ip.a[i] * x);
        out = x < ip.u[i] ? 0 : 1;
        break;
    case kAddition:
        t1 = x;
        break;
    case kDoubleGaussian: {
        const double v1 = ip.a[i] * (x - ip.u[i]), v2 = ip.a[i] * (x - ip.b[i]);
        t1 = exp(-(v1 * v1));
        t2 = exp(-(v2 * v2));
        break;
    }
    default:
        t1 = 0.0;
    }
}

// f from the combined product (multiplicative) or sum (additive).
__device__ __forceinline__ double pg_outer(int fid, int d, const IntegrandParams &ip, double A, double A2, int nout)
{
    switch (fid) {
    case kOscillatory: return cos(fma(6.283185307179586476925286766559, ip.u[0], A));
    case kCornerPeak: {
        const double b = 1.0 + A;
        double r = 1.0;
        for (int e = 0; e <= d; ++e) r *= b;
        return 1.0 / r;
    }
    case kAddition: return A;
    case kDiscontinuous: return nout == 0 ? A : 0.0;
    case kDoubleGaussian: return A + A2;
    default: return A;   // Gaussian, C0, product peak
    }
}

__device__ __forceinline__ int pair_index(int i, int j, int d)
{
    return i * (2 * d - i - 1) / 2 + (j - i - 1);   // pairs i < j in row-major order
}

__global__ void __launch_bounds__(kPgWarps * 32)
    pagani_evaluate_sep_kernel(const PgRule R, const IntegrandParams ip, int fid, long long n,
                               const double *__restrict__ lo, const double *__restrict__ len, double *__restrict__ I,
                               double *__restrict__ E, int *__restrict__ axis)
{
    __shared__ double fax[kPgWarps][kPgAxisPts];
    __shared__ PgAxisTab tabs[kPgWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, d = R.d;
    const bool mult = pg_mult(fid);
    const int npairs = d * (d - 1) / 2;
    PgAxisTab &T = tabs[warp];
    for (long long r = (long long)blockIdx.x * kPgWarps + warp; r < n; r += (long long)gridDim.x * kPgWarps) {
        const double *rlo = lo + r * d, *rlen = len + r * d;
        for (int e = lane; e < d * 9; e += 32) {
            const int i = e / 9, k = e - i * 9;
            const double lv = k == 0 ? 0.0 : (k <= 2 ? R.l2 : k <= 4 ? R.l3 : k <= 6 ? R.l4 : R.l5);
            const double u = (k & 1) || k == 0 ? lv : -lv;
            const double x = rlo[i] + 0.5 * rlen[i] * (1.0 + u);
            pg_terms(fid, ip, i, x, T.t1[i][k], T.t2[i][k], T.out[i][k]);
        }
        __syncwarp();
        // centre combinations over all axes, all but one, all but a pair
        for (int e = lane; e < 1 + d + npairs; e += 32) {
            int skip_i = -1, skip_j = -1;
            if (e >= 1 && e <= d) {
                skip_i = e - 1;
            } else if (e > d) {
                int pr = e - 1 - d, i = 0;
                while (pr >= d - 1 - i) {
                    pr -= d - 1 - i;
                    ++i;
                }
                skip_i = i;
                skip_j = i + 1 + pr;
            }
            double c1 = mult ? 1.0 : 0.0, c2 = mult ? 1.0 : 0.0;
            int no = 0;
            for (int i = 0; i < d; ++i) {
                if (i == skip_i || i == skip_j) continue;
                c1 = mult ? c1 * T.t1[i][0] : c1 + T.t1[i][0];
                c2 = mult ? c2 * T.t2[i][0] : c2 + T.t2[i][0];
                no += T.out[i][0];
            }
            if (e == 0) {
                T.all1 = c1;
                T.all2 = c2;
                T.nout_all = no;
            } else if (e <= d) {
                T.ex1[e - 1] = c1;
                T.ex2[e - 1] = c2;
                T.nout_ex1[e - 1] = no;
            } else {
                T.px1[e - 1 - d] = c1;
                T.px2[e - 1 - d] = c2;
                T.nout_px[e - 1 - d] = no;
            }
        }
        __syncwarp();
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
        for (int p = lane; p < R.n; p += 32) {
            double A, A2;
            int no, cls;
            if (p == 0) {
                A = T.all1;
                A2 = T.all2;
                no = T.nout_all;
                cls = 1;
            } else if (p < R.base4) {
                const bool c3 = p >= R.base3;
                const int q = c3 ? p - R.base3 : p - 1, k = q >> 1, idx = (c3 ? 3 : 1) + (q & 1);
                A = mult ? T.ex1[k] * T.t1[k][idx] : T.ex1[k] + T.t1[k][idx];
                A2 = mult ? T.ex2[k] * T.t2[k][idx] : 0.0;
                no = T.nout_ex1[k] + T.out[k][idx];
                cls = c3 ? 3 : 2;
            } else if (p < R.base5) {
                const int q = p - R.base4, sg = q & 3;
                int pair = q >> 2, i = 0;
                while (pair >= d - 1 - i) {
                    pair -= d - 1 - i;
                    ++i;
                }
                const int j = i + 1 + pair, ii = 5 + ((sg >> 1) & 1), ij = 5 + (sg & 1), pi = pair_index(i, j, d);
                A = mult ? T.px1[pi] * (T.t1[i][ii] * T.t1[j][ij]) : T.px1[pi] + (T.t1[i][ii] + T.t1[j][ij]);
                A2 = mult ? T.px2[pi] * (T.t2[i][ii] * T.t2[j][ij]) : 0.0;
                no = T.nout_px[pi] + T.out[i][ii] + T.out[j][ij];
                cls = 4;
            } else {
                const int b = p - R.base5;
                A = mult ? 1.0 : 0.0;
                A2 = mult ? 1.0 : 0.0;
                no = 0;
                for (int i = 0; i < d; ++i) {
                    const int idx = 7 + ((b >> i) & 1);
                    A = mult ? A * T.t1[i][idx] : A + T.t1[i][idx];
                    A2 = mult ? A2 * T.t2[i][idx] : A2;
                    no += T.out[i][idx];
                }
                cls = 5;
            }
            const double f = pg_outer(fid, d, ip, A, A2, no);
            if (cls == 5) s4 += f;
            else if (cls == 4) s3 += f;
            else if (cls == 3) s2 += f;
            else if (cls == 2) s1 += f;
            else s0 += f;
            if (p < R.base4) fax[warp][p] = f;
        }
        double S[5] = {s0, s1, s2, s3, s4};
#pragma unroll
        for (int k = 0; k < 5; ++k)
            for (int o = 16; o > 0; o >>= 1) S[k] += __shfl_xor_sync(0xffffffffu, S[k], o);
        __syncwarp();
        if (lane == 0) finish_region(R, S, fax[warp], rlen, I + r, E + r, axis + r);
        __syncwarp();   // the next region reuses the tables and fax
    }
}

__global__ void __launch_bounds__(kPgWarps * 32)
    pagani_evaluate_kernel(const PgRule R, const IntegrandParams ip, int fid, long long n, const double *__restrict__ lo,
                           const double *__restrict__ len, double *__restrict__ I, double *__restrict__ E,
                           int *__restrict__ axis)
{
    __shared__ double fax[kPgWarps][kPgAxisPts];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, d = R.d;
    for (long long r = (long long)blockIdx.x * kPgWarps + warp; r < n; r += (long long)gridDim.x * kPgWarps) {
        const double *rlo = lo + r * d, *rlen = len + r * d;
        double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int p = lane; p < R.n; p += 32) {
            double u[kDMax], x[kDMax];
            const int cls = rule_point(R, p, u);
            for (int i = 0; i < d; ++i) x[i] = rlo[i] + 0.5 * rlen[i] * (1.0 + u[i]);
            const double f = eval64(fid, d, ip, x);
            S[0] += cls == 1 ? f : 0.0;
            S[1] += cls == 2 ? f : 0.0;
            S[2] += cls == 3 ? f : 0.0;
            S[3] += cls == 4 ? f : 0.0;
            S[4] += cls == 5 ? f : 0.0;
            if (p < R.base5 && p < R.base4) fax[warp][p] = f;
        }
#pragma unroll
        for (int k = 0; k < 5; ++k)
            for (int o = 16; o > 0; o >>= 1) S[k] += __shfl_xor_sync(0xffffffffu, S[k], o);
        __syncwarp();
        if (lane == 0) finish_region(R, S, fax[warp], rlen, I + r, E + r, axis + r);
        __syncwarp();   // the next region reuses fax
    }
}

// ------------------------------------------------------------------------------ adaptive steps
// flag[r] = 1 when region r is split (E_r > thr V_r), else its I_r, E_r go to done[0..1].
__global__ void pagani_classify_kernel(long long n, int d, const double *__restrict__ len, const double *__restrict__ I,
                                       const double *__restrict__ E, double thr, int *__restrict__ flag,
                                       double *__restrict__ done)
{
    double sI = 0.0, sE = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        double vol = 1.0;
        for (int i = 0; i < d; ++i) vol *= len[r * d + i];
        const bool fin = E[r] <= thr * vol;
        flag[r] = fin ? 0 : 1;
        if (fin) {
            sI += I[r];
            sE += E[r];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sI += __shfl_xor_sync(0xffffffffu, sI, o);
        sE += __shfl_xor_sync(0xffffffffu, sE, o);
    }
    if ((threadIdx.x & 31) == 0 && (sI != 0.0 || sE != 0.0)) {
        atomicAdd(&done[0], sI);
        atomicAdd(&done[1], sE);
    }
}

// Exclusive scan of flag within blocks of kScanBlock: local offsets and block totals.
__global__ void __launch_bounds__(kScanBlock) scan_blocks_kernel(long long n, const int *__restrict__ flag,
                                                                 int *__restrict__ local, int *__restrict__ block_sum)
{
    __shared__ int wsum[kScanBlock / 32];
    const long long r = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v = r < n ? flag[r] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int before = (warp ? wsum[warp - 1] : 0) + x - v;
    if (r < n) local[r] = before;
    if (threadIdx.x == kScanBlock - 1) block_sum[blockIdx.x] = wsum[31];
}

// Exclusive scan of the block totals in one block (sequential runs per thread); total to *count.
__global__ void __launch_bounds__(kScanBlock) scan_totals_kernel(int nb, int *__restrict__ block_sum,
                                                                 long long *__restrict__ count)
{
    __shared__ int part[kScanBlock];
    const int per = (nb + kScanBlock - 1) / kScanBlock;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += block_sum[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < kScanBlock; ++t) {
            const int v = part[t];
            part[t] = run;
            run += v;
        }
        *count = run;
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        const int v = block_sum[b];
        block_sum[b] = run;
        run += v;
    }
}

// Children of every split region: lower half at 2 k, upper half at 2 k + 1, k its rank.
__global__ void pagani_split_kernel(long long n, int d, const double *__restrict__ lo, const double *__restrict__ len,
                                    const int *__restrict__ axis, const int *__restrict__ flag,
                                    const int *__restrict__ local, const int *__restrict__ block_off,
                                    double *__restrict__ lo2, double *__restrict__ len2)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        if (!flag[r]) continue;
        const long long k = (long long)local[r] + block_off[r / kScanBlock];
        const int ax = axis[r];
        for (int h = 0; h < 2; ++h) {
            double *cl = lo2 + (2 * k + h) * d, *cn = len2 + (2 * k + h) * d;
            for (int i = 0; i < d; ++i) {
                cl[i] = lo[r * d + i];
                cn[i] = len[r * d + i];
            }
            cn[ax] *= 0.5;
            if (h) cl[ax] += cn[ax];
        }
    }
}

__global__ void pagani_init_kernel(long long n, int d, int split, double *__restrict__ lo, double *__restrict__ len)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        long long t = r;
        for (int i = 0; i < d; ++i) {
            const int c = (int)(t % split);
            t /= split;
            lo[r * d + i] = (double)c / split;
            len[r * d + i] = 1.0 / split;
        }
    }
}

__global__ void sum2_kernel(long long n, const double *__restrict__ a, const double *__restrict__ b,
                            double *__restrict__ out)
{
    double sa = 0.0, sb = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        sa += a[r];
        sb += b[r];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], sa);
        atomicAdd(&out[1], sb);
    }
}

int num_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

int pagani_prepare(int fid, const double *params, int d, IntegrandParams &ip)
{
    if (d < 2 || d > MCUBES_DMAX) return MCUBES_ERR_UNSUPPORTED_DIM;
    Problem pb;
    const int st = prepare(fid, params, d, 1000, 0, 0, 0, 0, MCUBES_FP64, pb);
    if (st) return st;
    ip = pb.P.ip;
    return MCUBES_OK;
}

int launch_evaluate(const PgRule &R, const IntegrandParams &ip, int fid, long long n, const double *lo,
                    const double *len, double *I, double *E, int *axis, cudaStream_t s)
{
    if (n <= 0) return MCUBES_OK;
    const int sms = num_sms();
    if (sms <= 0) return cuda_status(cudaErrorNoDevice);
    const long long blocks = std::min<long long>((n + kPgWarps - 1) / kPgWarps, (long long)sms * 16);
    if (fid != kRotatedGaussian && fid != kConstant)
        pagani_evaluate_sep_kernel<<<(unsigned)blocks, kPgWarps * 32, 0, s>>>(R, ip, fid, n, lo, len, I, E, axis);
    else
        pagani_evaluate_kernel<<<(unsigned)blocks, kPgWarps * 32, 0, s>>>(R, ip, fid, n, lo, len, I, E, axis);
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" int mcubes_pagani_rule_points(int d)
{
    if (d < 2 || d > MCUBES_DMAX) return 0;
    return make_rule(d).n;
}

extern "C" int mcubes_pagani_evaluate_dev(int integrand_id, const double *params, int d, int64_t n_regions,
                                          const double *d_lo, const double *d_len, double *d_I, double *d_E,
                                          int32_t *d_axis, void *stream)
{
    if (n_regions < 0 || (n_regions > 0 && (!d_lo || !d_len || !d_I || !d_E || !d_axis))) return MCUBES_ERR_INVALID_ARG;
    IntegrandParams ip;
    int st = pagani_prepare(integrand_id, params, d, ip);
    if (st) return st;
    return launch_evaluate(make_rule(d), ip, integrand_id, n_regions, d_lo, d_len, d_I, d_E, d_axis,
                           (cudaStream_t)stream);
}

extern "C" int mcubes_pagani_integrate(int integrand_id, const double *params, int d, double rel_tol, int max_iters,
                                       int64_t max_regions, int init_split, mcubes_pagani_result *out)
{
    if (!out) return MCUBES_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    if (!(rel_tol > 0.0) || max_iters < 1 || max_regions < 1 || init_split < 1) return MCUBES_ERR_INVALID_ARG;
    IntegrandParams ip;
    int st = pagani_prepare(integrand_id, params, d, ip);
    if (st) return st;
    long long na = 1;
    for (int i = 0; i < d; ++i) {
        na *= init_split;
        if (na > max_regions) return MCUBES_ERR_INVALID_ARG;
    }
    if (max_regions > (1ll << 31) - 1) return MCUBES_ERR_INVALID_ARG;
    const PgRule R = make_rule(d);
    const long long cap = max_regions;
    const long long nb_max = (cap + kScanBlock - 1) / kScanBlock;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t rb = sizeof(double) * (size_t)cap * d;
    const size_t bytes = 4 * al(rb) + 2 * al(sizeof(double) * cap) + 3 * al(sizeof(int) * cap) +
                         al(sizeof(int) * nb_max) + al(sizeof(double) * 4) + al(sizeof(long long));
    char *mem = nullptr;
    if ((st = cuda_status(mc_malloc((void **)&mem, bytes)))) return st;
    char *q = mem;
    auto take = [&](size_t b) { char *r = q; q += al(b); return r; };
    double *lo[2] = {(double *)take(rb), (double *)take(rb)};
    double *len[2] = {(double *)take(rb), (double *)take(rb)};
    double *dI = (double *)take(sizeof(double) * cap), *dE = (double *)take(sizeof(double) * cap);
    int *dax = (int *)take(sizeof(int) * cap), *dflag = (int *)take(sizeof(int) * cap);
    int *dlocal = (int *)take(sizeof(int) * cap), *dblk = (int *)take(sizeof(int) * nb_max);
    double *dsums = (double *)take(sizeof(double) * 4);   // [0..1] finished I, E; [2..3] active I, E
    long long *dcount = (long long *)take(sizeof(long long));
    cudaStream_t s = nullptr;
    auto finish = [&](int code) {
        if (s) cudaStreamDestroy(s);
        cudaFree(mem);
        return code;
    };
    if ((st = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)))) return finish(st);
    const int sms = std::max(1, num_sms());
    auto grid_for = [&](long long n, int threads) {
        return (unsigned)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, (long long)sms * 8));
    };
    pagani_init_kernel<<<grid_for(na, 256), 256, 0, s>>>(na, d, init_split, lo[0], len[0]);
    if ((st = cuda_status(cudaGetLastError()))) return finish(st);
    if ((st = cuda_status(cudaMemsetAsync(dsums, 0, sizeof(double) * 4, s)))) return finish(st);
    int cur = 0, it = 0, status = 1;
    double evaluated = 0.0, I_tot = 0.0, E_tot = 0.0;
    double h[4];
    while (it < max_iters) {
        ++it;
        if ((st = launch_evaluate(R, ip, integrand_id, na, lo[cur], len[cur], dI, dE, dax, s))) return finish(st);
        evaluated += (double)na;
        if ((st = cuda_status(cudaMemsetAsync(dsums + 2, 0, sizeof(double) * 2, s)))) return finish(st);
        sum2_kernel<<<grid_for(na, 256), 256, 0, s>>>(na, dI, dE, dsums + 2);
        if ((st = cuda_status(cudaGetLastError()))) return finish(st);
        if ((st = cuda_status(cudaMemcpyAsync(h, dsums, sizeof(h), cudaMemcpyDeviceToHost, s)))) return finish(st);
        if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
        I_tot = h[0] + h[2];
        E_tot = h[1] + h[3];
        if (!std::isfinite(I_tot) || !std::isfinite(E_tot)) return finish(MCUBES_ERR_NONFINITE);
        if (E_tot <= rel_tol * std::fabs(I_tot)) {
            status = 0;
            break;
        }
        pagani_classify_kernel<<<grid_for(na, 256), 256, 0, s>>>(na, d, len[cur], dI, dE, rel_tol * std::fabs(I_tot),
                                                                 dflag, dsums);
        const long long nb = (na + kScanBlock - 1) / kScanBlock;
        scan_blocks_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(na, dflag, dlocal, dblk);
        scan_totals_kernel<<<1, kScanBlock, 0, s>>>((int)nb, dblk, dcount);
        if ((st = cuda_status(cudaGetLastError()))) return finish(st);
        long long keep = 0;
        if ((st = cuda_status(cudaMemcpyAsync(&keep, dcount, sizeof(long long), cudaMemcpyDeviceToHost, s))))
            return finish(st);
        if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
        if (2 * keep > cap) {
            status = 2;
            break;
        }
        if (keep == 0) {
            if ((st = cuda_status(cudaMemcpyAsync(h, dsums, sizeof(double) * 2, cudaMemcpyDeviceToHost, s))))
                return finish(st);
            if ((st = cuda_status(cudaStreamSynchronize(s)))) return finish(st);
            I_tot = h[0];
            E_tot = h[1];
            na = 0;
            status = E_tot <= rel_tol * std::fabs(I_tot) ? 0 : 1;
            break;
        }
        pagani_split_kernel<<<grid_for(na, 256), 256, 0, s>>>(na, d, lo[cur], len[cur], dax, dflag, dlocal, dblk,
                                                              lo[1 - cur], len[1 - cur]);
        if ((st = cuda_status(cudaGetLastError()))) return finish(st);
        cur = 1 - cur;
        na = 2 * keep;
    }
    out->estimate = I_tot;
    out->error = E_tot;
    out->regions_evaluated = (int64_t)evaluated;
    out->iterations = it;
    out->status = status;
    out->active_regions = na;
    return finish(MCUBES_OK);
}
