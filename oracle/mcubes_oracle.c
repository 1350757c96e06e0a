/*
 * m-Cubes CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 restatement of one m-Cubes iteration:
 *   - the V-Sample kernel of the paper (Sec. 3.2, Algorithm 2): stratified sub-cube
 *     sampling through the VEGAS importance grid, integrand evaluation, per-cube mean
 *     and variance, bin contributions;
 *   - the grid refinement that m-Cubes inherits from VEGAS (Lepage 1978, cited in Sec. 3.2);
 *   - the benchmark integrands of Sec. 5 (Eq. 1-6, the addition integrand of Sec. 5.3)
 *     written as their Genz families;
 *   - the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3", SC'11) that replaces the paper's unspecified
 *     "simple custom-made random generator" (Sec. 4).
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load this file. It shares no code, header, table or constant generator with the CUDA
 * library; the two agree only through the documented interface numbers (integrand ids,
 * 500 bins per axis, Philox counter layout), which each side spells out itself.
 *
 * Readings of points the paper leaves open are stated next to the code that takes them.
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math: the FP32-eval
 * map below must round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ND 500  /* bins per axis, Algorithm 2 inputs B[500*d], C[500*d]; Sec. 3.2 */
#define ORC_DMAX 16

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,
    ORC_ERR_DIM = 2,
    ORC_ERR_INTEGRAND = 3,
};

/* Integrand ids: the Genz families behind Eq. 1-6 plus the addition integrand and a
 * constant. Parameters are a[0..d-1] followed by u[0..d-1]. */
enum {
    ORC_OSCILLATORY = 0,  /* cos(2 pi u_1 + sum a_i x_i)          ; Eq. 1 has a_i = i, u_1 = 0 */
    ORC_PRODUCT_PEAK = 1, /* prod (a_i^-2 + (x_i - u_i)^2)^-1      ; Eq. 2 has a_i = 50, u_i = 1/2 */
    ORC_CORNER_PEAK = 2,  /* (1 + sum a_i x_i)^-(d+1)              ; Eq. 3 has a_i = i */
    ORC_GAUSSIAN = 3,     /* exp(-sum a_i^2 (x_i - u_i)^2)         ; Eq. 4 has a_i = 25, u_i = 1/2 */
    ORC_C0 = 4,           /* exp(-sum a_i |x_i - u_i|)             ; Eq. 5 has a_i = 10, u_i = 1/2 */
    ORC_DISCONTINUOUS = 5,/* exp(sum a_i x_i) if x_i < u_i for all i, else 0
                             ; Eq. 6 has a_i = i + 4, u_i = (3 + i)/10 */
    ORC_ADDITION = 6,     /* sum x_i                                ; Sec. 5.3 */
    ORC_CONSTANT = 7,     /* a_1                                    ; exactness check */
    ORC_DOUBLE_GAUSSIAN = 8, /* exp(-sum a_i^2 (x_i-u_i)^2) + exp(-sum a_i^2 (x_i-1+u_i)^2): two peaks
                                mirrored through the centre (the learned proposal's test case) */
    ORC_ROTATED_GAUSSIAN = 9,/* exp(-(x-c)^T M (x-c)); params are M (d x d, row-major) then c (d) */
    ORC_N_INTEGRANDS = 10
};

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. SC'11): 10 rounds of the 4-word Philox S-box with the     */
/* published multipliers and Weyl key increments.                                        */
/* ------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------------------ */
/* Stratification (Sec. 3.2): split [0,1]^d into m = g^d sub-cubes so that a 2-point MC   */
/* estimate runs in each while about n samples are drawn.                                */
/* Reading: g is the largest integer with 2 g^d <= n; p = max(2, floor(n / m)).          */
/* ------------------------------------------------------------------------------------ */
static int pow_leq(int64_t g, int d, int64_t limit)  /* 1 if g^d <= limit, no overflow */
{
    int64_t v = 1;
    for (int i = 0; i < d; ++i) {
        if (v > limit / g) return 0;
        v *= g;
    }
    return v <= limit;
}

int orc_stratify(int d, int64_t n, int64_t *g_out, int64_t *m_out, int64_t *p_out)
{
    if (d < 1 || d > ORC_DMAX) return ORC_ERR_DIM;
    if (n < 2) return ORC_ERR_ARG;
    int64_t half = n / 2;            /* 2 g^d <= n  <=>  g^d <= floor(n/2) */
    int64_t lo = 1, hi = half;       /* g = 1 always satisfies it */
    while (lo < hi) {                /* largest g with g^d <= half */
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (pow_leq(mid, d, half)) lo = mid; else hi = mid - 1;
    }
    int64_t m = 1;
    for (int i = 0; i < d; ++i) m *= lo;
    if (m > (int64_t)0xFFFFFFFFll) return ORC_ERR_ARG; /* cube index is one counter word */
    int64_t p = n / m;
    if (p < 2) p = 2;
    *g_out = lo; *m_out = m; *p_out = p;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Integrands (Sec. 5, Eq. 1-6; addition Sec. 5.3), evaluated in FP64.                    */
/* fp32_cut: take the discontinuous family's cut decision in single precision, as the     */
/* FP32-eval variant does (the decision is made in the precision that forms the point).   */
/* ------------------------------------------------------------------------------------ */
double orc_integrand(int id, int d, const double *par, const double *x, int fp32_cut)
{
    const double *a = par, *u = par + d;
    const double two_pi = 6.283185307179586476925286766559;
    double s = 0.0, prod = 1.0;
    switch (id) {
    case ORC_OSCILLATORY:
        for (int i = 0; i < d; ++i) s += a[i] * x[i];
        return cos(two_pi * u[0] + s);
    case ORC_PRODUCT_PEAK:
        for (int i = 0; i < d; ++i) {
            double t = x[i] - u[i];
            prod *= 1.0 / (1.0 / (a[i] * a[i]) + t * t);
        }
        return prod;
    case ORC_CORNER_PEAK:
        for (int i = 0; i < d; ++i) s += a[i] * x[i];
        return pow(1.0 + s, -(double)(d + 1));
    case ORC_GAUSSIAN:
        for (int i = 0; i < d; ++i) {
            double t = x[i] - u[i];
            s += a[i] * a[i] * t * t;
        }
        return exp(-s);
    case ORC_C0:
        for (int i = 0; i < d; ++i) s += a[i] * fabs(x[i] - u[i]);
        return exp(-s);
    case ORC_DISCONTINUOUS:
        /* Reading of Eq. 6: the cut applies on every axis. */
        for (int i = 0; i < d; ++i) {
            int inside = fp32_cut ? ((float)x[i] < (float)u[i]) : (x[i] < u[i]);
            if (!inside) return 0.0;
            s += a[i] * x[i];
        }
        return exp(s);
    case ORC_ADDITION:
        for (int i = 0; i < d; ++i) s += x[i];
        return s;
    case ORC_CONSTANT:
        return a[0];
    case ORC_DOUBLE_GAUSSIAN: {
        double s2 = 0.0;
        for (int i = 0; i < d; ++i) {
            double t1 = x[i] - u[i], t2 = x[i] - (1.0 - u[i]);
            s += a[i] * a[i] * t1 * t1;
            s2 += a[i] * a[i] * t2 * t2;
        }
        return exp(-s) + exp(-s2);
    }
    case ORC_ROTATED_GAUSSIAN: {
        const double *M = par, *c = par + (size_t)d * d;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) s += (x[i] - c[i]) * M[i * d + j] * (x[j] - c[j]);
        return exp(-s);
    }
    default:
        return NAN;
    }
}

/* Neumaier-compensated running sum: value = sum + comp. */
typedef struct { double sum, comp; } orc_acc;

static void acc_add(orc_acc *acc, double v)
{
    double t = acc->sum + v;
    if (fabs(acc->sum) >= fabs(v)) acc->comp += (acc->sum - t) + v;
    else acc->comp += (v - t) + acc->sum;
    acc->sum = t;
}

/* ------------------------------------------------------------------------------------ */
/* Uniform draws. Philox counter for (cube t, sample q, call j, iteration it, job):       */
/* ctr = (t, q, (it << 16) | j, job), key = (seed mod 2^32, seed >> 32).                  */
/*   FP64 layout: call j serves dims 2j (words 0,1) and 2j+1 (words 2,3);                 */
/*                u = ((w_hi mod 2^20) * 2^32 + w_lo) * 2^-52.                              */
/*   FP32 layout: call j serves dims 4j..4j+3, one word each; u = (w mod 2^23) * 2^-23.    */
/* ------------------------------------------------------------------------------------ */
static void draw_uniforms(int fp32, int d, uint32_t t, uint32_t q, int it, uint32_t job,
                          uint64_t seed, double *u_out)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    uint32_t w[4];
    if (!fp32) {
        for (int j = 0; 2 * j < d; ++j) {
            uint32_t ctr[4] = { t, q, ((uint32_t)it << 16) | (uint32_t)j, job };
            orc_philox4x32_10(ctr, key, w);
            for (int h = 0; h < 2 && 2 * j + h < d; ++h) {
                uint64_t bits = ((uint64_t)(w[2 * h] & 0xFFFFFu) << 32) | (uint64_t)w[2 * h + 1];
                u_out[2 * j + h] = (double)bits * 0x1p-52;
            }
        }
    } else {
        for (int j = 0; 4 * j < d; ++j) {
            uint32_t ctr[4] = { t, q, ((uint32_t)it << 16) | (uint32_t)j, job };
            orc_philox4x32_10(ctr, key, w);
            for (int h = 0; h < 4 && 4 * j + h < d; ++h)
                u_out[4 * j + h] = (double)(w[h] & 0x7FFFFFu) * 0x1p-23;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* One V-Sample pass (Algorithm 2) over sub-cubes [t0, t1).                              */
/*                                                                                        */
/* Sub-cube t has digits c_i = floor(t / g^i) mod g (axis 0 fastest). For each of its p   */
/* samples and each axis i: yn = (c_i + u) * R with R = nd / g, capped below nd; the bin  */
/* is k = floor(yn), the offset in the bin delta = yn - k, the point                       */
/* x_i = B_i[k] + Delta_i[k] * delta with Delta_i[k] = B_i[k+1] - B_i[k], and the weight   */
/* of the sample is w = f(x) * prod_i (nd * Delta_i[k]).                                  */
/*   mode 0 (FP64): every step above in FP64.                                              */
/*   mode 1 (FP32-eval): the point is formed in single precision exactly as written above  */
/*     (u, c_i + u, the product with R, the cap, the bin, delta, and one fused multiply-   */
/*     add with the grid values rounded to single); the integrand and the Jacobian are     */
/*     then evaluated in FP64 at that point.                                               */
/* Per sub-cube (Algorithm 2, UpdateVariance; reading): I_t = S1/p and                     */
/*   V_t = max(0, S2 - S1^2/p) / (p (p-1)), with S1 = sum w and S2 = sum w^2.               */
/* Bin contributions (Algorithm 2, AtomicAdd into C): when adjust is set, every sample     */
/*   adds w^2 to C_i[k_i] on every axis.                                                   */
/* Outputs: sums of I_t and V_t over the range (compensated: sum and remainder), C          */
/* accumulated (C is d*nd doubles, C_comp its compensation, either may be NULL when adjust  */
/* is 0), optional per-cube I_t, V_t for t in [t0, t1).                                   */
/* ------------------------------------------------------------------------------------ */
int orc_vsample(int id, int d, const double *par, int64_t n, uint64_t seed, int it,
                uint32_t job, int mode, int adjust, const double *B,
                int64_t t0, int64_t t1,
                double *sumI, double *sumV, double *C, double *C_comp,
                double *cubeI, double *cubeV)
{
    int64_t g, m, p;
    int st = orc_stratify(d, n, &g, &m, &p);
    if (st) return st;
    if (id < 0 || id >= ORC_N_INTEGRANDS) return ORC_ERR_INTEGRAND;
    if (mode != 0 && mode != 1) return ORC_ERR_ARG;
    if (t0 < 0 || t1 > m || t0 > t1) return ORC_ERR_ARG;
    if (it < 0 || it > 0xFFFF) return ORC_ERR_ARG;

    const int nd = ORC_ND;
    const double R = (double)nd / (double)g;
    const double ycap = nextafter((double)nd, 0.0);        /* largest double below nd */
    const float R32 = (float)R;
    const float ycap32 = nextafterf((float)nd, 0.0f);     /* largest float below nd */

    orc_acc accI = {0, 0}, accV = {0, 0};
    double u[ORC_DMAX], x[ORC_DMAX];
    int kbin[ORC_DMAX];

    for (int64_t t = t0; t < t1; ++t) {
        int64_t c[ORC_DMAX];
        int64_t rest = t;
        for (int i = 0; i < d; ++i) { c[i] = rest % g; rest /= g; }

        orc_acc s1 = {0, 0}, s2 = {0, 0};
        for (int64_t q = 0; q < p; ++q) {
            draw_uniforms(mode == 1, d, (uint32_t)t, (uint32_t)q, it, job, seed, u);
            double J = 1.0;
            for (int i = 0; i < d; ++i) {
                const double *Bi = B + (size_t)i * (nd + 1);
                int k;
                if (mode == 0) {
                    double yn = ((double)c[i] + u[i]) * R;
                    if (yn > ycap) yn = ycap;
                    k = (int)floor(yn);
                    double delta = yn - (double)k;
                    double width = Bi[k + 1] - Bi[k];
                    x[i] = fma(width, delta, Bi[k]);
                    J *= (double)nd * width;
                } else {
                    float s = (float)c[i] + (float)u[i];
                    float yn = s * R32;
                    if (yn > ycap32) yn = ycap32;
                    k = (int)floorf(yn);
                    float delta = yn - (float)k;
                    double width = Bi[k + 1] - Bi[k];
                    float x32 = fmaf((float)width, delta, (float)Bi[k]);
                    x[i] = (double)x32;
                    J *= (double)nd * width;
                }
                kbin[i] = k;
            }
            double f = orc_integrand(id, d, par, x, mode == 1);
            double w = f * J;
            acc_add(&s1, w);
            acc_add(&s2, w * w);
            if (adjust && C) {
                for (int i = 0; i < d; ++i) {
                    size_t idx = (size_t)i * nd + (size_t)kbin[i];
                    if (C_comp) {
                        orc_acc a = { C[idx], C_comp[idx] };
                        acc_add(&a, w * w);
                        C[idx] = a.sum; C_comp[idx] = a.comp;
                    } else {
                        C[idx] += w * w;
                    }
                }
            }
        }
        double S1 = s1.sum + s1.comp, S2 = s2.sum + s2.comp;
        double It = S1 / (double)p;
        double num = S2 - S1 * S1 / (double)p;
        if (num < 0.0) num = 0.0;
        double Vt = num / ((double)p * (double)(p - 1));
        acc_add(&accI, It);
        acc_add(&accV, Vt);
        if (cubeI) cubeI[t - t0] = It;
        if (cubeV) cubeV[t - t0] = Vt;
    }
    sumI[0] = accI.sum; sumI[1] = accI.comp;
    sumV[0] = accV.sum; sumV[1] = accV.comp;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Grid refinement (VEGAS, Lepage 1978; m-Cubes Sec. 3.2 delegates to it). Per axis:      */
/*  1. smooth:  d_0 = (C_0 + C_1)/2, d_k = (C_{k-1} + C_k + C_{k+1})/3,                    */
/*              d_{nd-1} = (C_{nd-2} + C_{nd-1})/2;                                         */
/*  2. D = sum d_k; if D is 0 (or not finite) the axis keeps its grid;                      */
/*  3. compress: rho = d_k / D, r_k = 0 if d_k = 0, 1 if rho = 1,                          */
/*              else ((1 - rho) / (-ln rho))^alpha;                                         */
/*  4. redistribute: R_0 = 0, R_{k+1} = R_k + r_k, S = R_nd; new boundary l (1..nd-1)      */
/*              sits where the running r-mass reaches l S / nd, linear inside the old bin:  */
/*              B'_l = B_k + Delta_k (l S/nd - R_k) / r_k with R_k <= l S/nd < R_{k+1}.      */
/*     B'_0 = 0, B'_nd = 1.                                                                 */
/* ------------------------------------------------------------------------------------ */
/* Step 3's damped weight of one bin with mass fraction 0 < rho <= 1 (1 at rho = 1). */
double orc_damp(double rho, double alpha)
{
    if (rho == 1.0) return 1.0;
    return pow((1.0 - rho) / (-log(rho)), alpha);
}

void orc_rebin(int d, const double *B, const double *C, double alpha, double *Bout)
{
    const int nd = ORC_ND;
    double dsm[ORC_ND], r[ORC_ND], Rc[ORC_ND + 1];
    for (int i = 0; i < d; ++i) {
        const double *Bi = B + (size_t)i * (nd + 1);
        const double *Ci = C + (size_t)i * nd;
        double *Bo = Bout + (size_t)i * (nd + 1);

        dsm[0] = (Ci[0] + Ci[1]) / 2.0;
        for (int k = 1; k < nd - 1; ++k) dsm[k] = (Ci[k - 1] + Ci[k] + Ci[k + 1]) / 3.0;
        dsm[nd - 1] = (Ci[nd - 2] + Ci[nd - 1]) / 2.0;

        double D = 0.0;
        for (int k = 0; k < nd; ++k) D += dsm[k];
        if (!(D > 0.0) || !isfinite(D)) {
            memmove(Bo, Bi, sizeof(double) * (nd + 1));
            continue;
        }
        for (int k = 0; k < nd; ++k) {
            double rho = dsm[k] / D;
            r[k] = dsm[k] == 0.0 ? 0.0 : orc_damp(rho, alpha);
        }
        Rc[0] = 0.0;
        for (int k = 0; k < nd; ++k) Rc[k + 1] = Rc[k] + r[k];
        double S = Rc[nd];

        double newB[ORC_ND + 1];
        newB[0] = 0.0;
        newB[nd] = 1.0;
        int k = 0;
        for (int l = 1; l < nd; ++l) {
            double T = (double)l * S / (double)nd;
            while (k < nd - 1 && !(Rc[k] <= T && T < Rc[k + 1] && r[k] > 0.0)) ++k;
            double width = Bi[k + 1] - Bi[k];
            /* Reading: the new boundary stays inside old bin k; rounding of the running
               sum can push the fraction a hair past 1, which is cut back to 1. */
            double frac = r[k] > 0.0 ? (T - Rc[k]) / r[k] : 0.0;
            if (frac > 1.0) frac = 1.0;
            if (frac < 0.0) frac = 0.0;
            newB[l] = Bi[k] + width * frac;
        }
        memcpy(Bo, newB, sizeof(double) * (nd + 1));
    }
}

/* Per-sample record of the V-Sample steps for sub-cubes [t0, t1): uniforms u, point x,
 * bin k, Jacobian J and weight w, laid out sample-major ((t - t0) * p + q). Lets tests
 * check each step of the map and the accumulation against library routines. */
int orc_sample_points(int id, int d, const double *par, int64_t n, uint64_t seed, int it,
                      uint32_t job, int mode, const double *B, int64_t t0, int64_t t1,
                      double *u_out, double *x_out, int32_t *k_out, double *J_out, double *w_out)
{
    int64_t g, m, p;
    int st = orc_stratify(d, n, &g, &m, &p);
    if (st) return st;
    if (t0 < 0 || t1 > m || t0 > t1 || it < 0 || it > 0xFFFF) return ORC_ERR_ARG;
    const int nd = ORC_ND;
    const double R = (double)nd / (double)g;
    const double ycap = nextafter((double)nd, 0.0);
    const float R32 = (float)R;
    const float ycap32 = nextafterf((float)nd, 0.0f);
    double u[ORC_DMAX], x[ORC_DMAX];
    size_t row = 0;
    for (int64_t t = t0; t < t1; ++t) {
        int64_t c[ORC_DMAX], rest = t;
        for (int i = 0; i < d; ++i) { c[i] = rest % g; rest /= g; }
        for (int64_t q = 0; q < p; ++q, ++row) {
            draw_uniforms(mode == 1, d, (uint32_t)t, (uint32_t)q, it, job, seed, u);
            double J = 1.0;
            for (int i = 0; i < d; ++i) {
                const double *Bi = B + (size_t)i * (nd + 1);
                int k;
                if (mode == 0) {
                    double yn = ((double)c[i] + u[i]) * R;
                    if (yn > ycap) yn = ycap;
                    k = (int)floor(yn);
                    double width = Bi[k + 1] - Bi[k];
                    x[i] = fma(width, yn - (double)k, Bi[k]);
                    J *= (double)nd * width;
                } else {
                    float s = (float)c[i] + (float)u[i];
                    float yn = s * R32;
                    if (yn > ycap32) yn = ycap32;
                    k = (int)floorf(yn);
                    double width = Bi[k + 1] - Bi[k];
                    x[i] = (double)fmaf((float)width, yn - (float)k, (float)Bi[k]);
                    J *= (double)nd * width;
                }
                if (u_out) u_out[row * d + i] = u[i];
                if (x_out) x_out[row * d + i] = x[i];
                if (k_out) k_out[row * d + i] = k;
            }
            double f = orc_integrand(id, d, par, x, mode == 1);
            if (J_out) J_out[row] = J;
            if (w_out) w_out[row] = f * J;
        }
    }
    return ORC_OK;
}

/* f at npts points (row-major npts x d), FP64. */
void orc_integrand_many(int id, int d, const double *par, int64_t npts, const double *X,
                        double *out)
{
    for (int64_t r = 0; r < npts; ++r) out[r] = orc_integrand(id, d, par, X + r * d, 0);
}

/* Uniform starting grid: B_i[k] = k / nd. */
void orc_uniform_grid(int d, double *B)
{
    for (int i = 0; i < d; ++i)
        for (int k = 0; k <= ORC_ND; ++k)
            B[(size_t)i * (ORC_ND + 1) + k] = (double)k / (double)ORC_ND;
}

/* ------------------------------------------------------------------------------------ */
/* Whole integration: itmax iterations, the first iter_adjust refine the grid (reading of */
/* the grid-adjust vs frozen split), then the iterations are combined by inverse-variance */
/* weighting (VEGAS convention; reading):                                                  */
/*   Ibar = sum(I_it / V_it) / sum(1 / V_it), sigma = sum(1 / V_it)^-1/2,                  */
/*   chi2/dof = sum (I_it - Ibar)^2 / V_it / (N - 1)  (0 when N = 1).                       */
/* Iterations with V_it = 0 (exact for the sampled points): Ibar is their mean, sigma 0,   */
/* chi2/dof 0.                                                                             */
/* Outputs: est[3] = {Ibar, sigma, chi2/dof}; iterI, iterV (itmax each, optional); B is    */
/* the starting grid on input (NULL: uniform) -- it is not modified.                       */
/* ------------------------------------------------------------------------------------ */
int orc_integrate(int id, int d, const double *par, int64_t n, int itmax, int iter_adjust,
                  uint64_t seed, uint32_t job, int mode, const double *B_in,
                  double *est, double *iterI, double *iterV)
{
    int64_t g, m, p;
    int st = orc_stratify(d, n, &g, &m, &p);
    if (st) return st;
    if (itmax < 1 || iter_adjust < 0 || iter_adjust > itmax || itmax > 0xFFFF) return ORC_ERR_ARG;

    const int nd = ORC_ND;
    size_t nb = (size_t)d * (nd + 1), nc = (size_t)d * nd;
    double *B = malloc(sizeof(double) * nb), *Bn = malloc(sizeof(double) * nb);
    double *C = malloc(sizeof(double) * nc), *Cc = malloc(sizeof(double) * nc);
    double *Is = malloc(sizeof(double) * itmax), *Vs = malloc(sizeof(double) * itmax);
    if (!B || !Bn || !C || !Cc || !Is || !Vs) {
        free(B); free(Bn); free(C); free(Cc); free(Is); free(Vs);
        return ORC_ERR_ARG;
    }
    if (B_in) memcpy(B, B_in, sizeof(double) * nb); else orc_uniform_grid(d, B);

    for (int it = 0; it < itmax; ++it) {
        int adjust = it < iter_adjust;
        memset(C, 0, sizeof(double) * nc);
        memset(Cc, 0, sizeof(double) * nc);
        double sI[2], sV[2];
        st = orc_vsample(id, d, par, n, seed, it, job, mode, adjust, B, 0, m, sI, sV, C, Cc, NULL, NULL);
        if (st) break;
        Is[it] = (sI[0] + sI[1]) / (double)m;
        Vs[it] = (sV[0] + sV[1]) / ((double)m * (double)m);
        if (adjust && it + 1 < itmax) {
            for (size_t e = 0; e < nc; ++e) C[e] += Cc[e];
            orc_rebin(d, B, C, 1.5, Bn);
            double *tmp = B; B = Bn; Bn = tmp;
        }
    }
    if (!st) {
        int nzero = 0;
        double zsum = 0.0;
        for (int it = 0; it < itmax; ++it) if (Vs[it] == 0.0) { ++nzero; zsum += Is[it]; }
        if (nzero > 0) {
            est[0] = zsum / nzero; est[1] = 0.0; est[2] = 0.0;
        } else {
            double sw = 0.0, swI = 0.0;
            for (int it = 0; it < itmax; ++it) { sw += 1.0 / Vs[it]; swI += Is[it] / Vs[it]; }
            double Ibar = swI / sw;
            double chi = 0.0;
            for (int it = 0; it < itmax; ++it) chi += (Is[it] - Ibar) * (Is[it] - Ibar) / Vs[it];
            est[0] = Ibar;
            est[1] = 1.0 / sqrt(sw);
            est[2] = itmax > 1 ? chi / (double)(itmax - 1) : 0.0;
        }
        if (iterI) memcpy(iterI, Is, sizeof(double) * itmax);
        if (iterV) memcpy(iterV, Vs, sizeof(double) * itmax);
    }
    free(B); free(Bn); free(C); free(Cc); free(Is); free(Vs);
    return st;
}

/* Grid after `iters` adjusting iterations (for per-iteration parity on adapted grids). */
int orc_adapted_grid(int id, int d, const double *par, int64_t n, int iters, uint64_t seed,
                     uint32_t job, int mode, double *B_out)
{
    int64_t g, m, p;
    int st = orc_stratify(d, n, &g, &m, &p);
    if (st) return st;
    const int nd = ORC_ND;
    size_t nb = (size_t)d * (nd + 1), nc = (size_t)d * nd;
    double *B = malloc(sizeof(double) * nb), *C = malloc(sizeof(double) * nc);
    double *Cc = malloc(sizeof(double) * nc);
    if (!B || !C || !Cc) { free(B); free(C); free(Cc); return ORC_ERR_ARG; }
    orc_uniform_grid(d, B);
    for (int it = 0; it < iters && !st; ++it) {
        memset(C, 0, sizeof(double) * nc);
        memset(Cc, 0, sizeof(double) * nc);
        double sI[2], sV[2];
        st = orc_vsample(id, d, par, n, seed, it, job, mode, 1, B, 0, m, sI, sV, C, Cc, NULL, NULL);
        for (size_t e = 0; e < nc; ++e) C[e] += Cc[e];
        if (!st) orc_rebin(d, B, C, 1.5, B_out), memcpy(B, B_out, sizeof(double) * nb);
    }
    if (!st) memcpy(B_out, B, sizeof(double) * nb);
    free(B); free(C); free(Cc);
    return st;
}
