/*
 * PAGANI oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain FP64 restatement of the paper's other workload, the PAGANI region evaluation
 * (Sec. 3.1, the PAGANI-kernel algorithm), and of a simple adaptive driver around it.
 *
 * Per region (low corner lo, side lengths len) the kernel evaluates a fully symmetric cubature
 * rule at f_eval points and returns an integral estimate, an error estimate and the axis to split.
 * The paper defers the rules themselves to PAGANI; the reading here is the published
 * Genz-Malik rule of degree 7 with its embedded rule of degree 5 (A. C. Genz, A. A. Malik,
 * "An adaptive algorithm for numerical integration over an n-dimensional rectangular region",
 * J. Comput. Appl. Math. 6 (1980)), on the reference cube [-1, 1]^d:
 *   generators (classes): 1: the centre; 2: +-l2 e_i; 3: +-l3 e_i; 4: +-l4 e_i +- l4 e_j (i < j);
 *                         5: (+-l5, ..., +-l5), all 2^d sign patterns;
 *   l2^2 = 9/70, l3^2 = l4^2 = 9/10, l5^2 = 9/19;
 *   f_eval = 1 + 4d + 2d(d-1) + 2^d points;
 *   degree 7: w1 = 2^d (12824 - 9120 d + 400 d^2)/19683, w2 = 2^d 980/6561,
 *             w3 = 2^d (1820 - 400 d)/19683, w4 = 2^d 200/19683, w5 = 6859/19683;
 *   degree 5: w1 = 2^d (729 - 950 d + 50 d^2)/729, w2 = 2^d 245/486,
 *             w3 = 2^d (265 - 100 d)/1458, w4 = 2^d 25/729, w5 = 0.
 * The paper's kernel accumulates five quadrature rules per region and takes the error from them;
 * the reading adds three lower-degree rules on the same points, from the moment conditions
 * (exact for 1 and x_i^2 on [-1, 1]^d, whose integrals are 2^d and 2^d / 3):
 *   R3a, degree 3 on classes 1, 2: w2 = 2^d / (6 l2^2), w1 = 2^d - 2 d w2;
 *   R3b, degree 3 on classes 1, 3: w3 = 2^d / (6 l3^2), w1 = 2^d - 2 d w3;
 *   R1, degree 1: w1 = 2^d (the centre).
 * Integral estimate I7 = (V / 2^d) sum_k w7_k S_k, with S_k the sum of f over class k and V the
 * region's volume. Error estimate from the differences of successive degrees,
 *   D7 = |R7 - R5|, D5 = max(|R5 - R3a|, |R5 - R3b|), D3 = max(|R3a - R1|, |R3b - R1|):
 * E = D7 when each difference is at most a quarter of the previous one (D7 <= D5 / 4 and
 * D5 <= D3 / 4: the rules are in their asymptotic range, where D7, the degree-5 rule's error,
 * bounds the degree-7 rule's), and E = max(D7, D5, D3) otherwise. Split axis: the largest fourth divided
 * difference |f(l2 e_i) + f(-l2 e_i) - 2 f(0) - (l2/l3)^2 (f(l3 e_i) + f(-l3 e_i) - 2 f(0))|,
 * with ties going to the longest side, then the lowest axis. Two differences tie when they are
 * within 1e-12 of the larger of them and of the largest |f| at the centre and axis points (below
 * that a fourth difference is rounding noise).
 *
 * Only the test-suite and the benchmark's CPU-baseline leg may load this file. It shares no
 * code with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PG_DMAX 16

double orc_integrand(int id, int d, const double *par, const double *x, int fp32_cut);

static double pg_lambda2(int k)
{
    switch (k) {
    case 2: return 9.0 / 70.0;
    case 3: return 9.0 / 10.0;
    case 4: return 9.0 / 10.0;
    default: return 9.0 / 19.0;
    }
}

int orc_gm_count(int d)
{
    if (d < 2 || d > PG_DMAX) return 0;
    return 1 + 4 * d + 2 * d * (d - 1) + (1 << d);
}

/* Rule weights per class 1..5 (index 0..4), degree 7 and degree 5, on [-1, 1]^d. */
/* The five rules' class weights on [-1, 1]^d: W[r][k] for rule r = R7, R5, R3a, R3b, R1 and
 * class k = 1..5 (index k - 1). */
void orc_gm_rules(int d, double *W /* 5 x 5 */);

void orc_gm_weights(int d, double *w7, double *w5)
{
    const double two_d = ldexp(1.0, d), dd = (double)d;
    w7[0] = two_d * (12824.0 - 9120.0 * dd + 400.0 * dd * dd) / 19683.0;
    w7[1] = two_d * 980.0 / 6561.0;
    w7[2] = two_d * (1820.0 - 400.0 * dd) / 19683.0;
    w7[3] = two_d * 200.0 / 19683.0;
    w7[4] = 6859.0 / 19683.0;
    w5[0] = two_d * (729.0 - 950.0 * dd + 50.0 * dd * dd) / 729.0;
    w5[1] = two_d * 245.0 / 486.0;
    w5[2] = two_d * (265.0 - 100.0 * dd) / 1458.0;
    w5[3] = two_d * 25.0 / 729.0;
    w5[4] = 0.0;
}

void orc_gm_rules(int d, double *W)
{
    const double two_d = ldexp(1.0, d);
    memset(W, 0, sizeof(double) * 25);
    orc_gm_weights(d, W, W + 5);
    W[2 * 5 + 1] = two_d / (6.0 * pg_lambda2(2));
    W[2 * 5 + 0] = two_d - 2.0 * d * W[2 * 5 + 1];
    W[3 * 5 + 2] = two_d / (6.0 * pg_lambda2(3));
    W[3 * 5 + 0] = two_d - 2.0 * d * W[3 * 5 + 2];
    W[4 * 5 + 0] = two_d;
}

/* The error estimate from the five rule values R[0..4] = R7, R5, R3a, R3b, R1 (see the header). */
double orc_pagani_error(const double *R)
{
    const double d7 = fabs(R[0] - R[1]);
    const double d5 = fmax(fabs(R[1] - R[2]), fabs(R[1] - R[3]));
    const double d3 = fmax(fabs(R[2] - R[4]), fabs(R[3] - R[4]));
    if (d7 <= 0.25 * d5 && d5 <= 0.25 * d3) return d7;
    return fmax(d7, fmax(d5, d3));
}

/* All rule points on [-1, 1]^d in the order centre, class 2 (axis-major, + then -), class 3,
 * class 4 (pairs i < j in row-major order; signs (+,+), (+,-), (-,+), (-,-)), class 5 (sign
 * pattern b: bit i set = negative on axis i, b = 0 .. 2^d - 1). U: count x d; cls: count. */
int orc_gm_points(int d, double *U, int *cls)
{
    const int n = orc_gm_count(d);
    if (!n) return 1;
    memset(U, 0, sizeof(double) * (size_t)n * d);
    int p = 0;
    cls[p++] = 1;
    for (int k = 2; k <= 3; ++k) {
        const double l = sqrt(pg_lambda2(k));
        for (int i = 0; i < d; ++i)
            for (int s = 0; s < 2; ++s) {
                U[(size_t)p * d + i] = s ? -l : l;
                cls[p++] = k;
            }
    }
    {
        const double l = sqrt(pg_lambda2(4));
        for (int i = 0; i < d; ++i)
            for (int j = i + 1; j < d; ++j)
                for (int s = 0; s < 4; ++s) {
                    U[(size_t)p * d + i] = (s & 2) ? -l : l;
                    U[(size_t)p * d + j] = (s & 1) ? -l : l;
                    cls[p++] = 4;
                }
    }
    {
        const double l = sqrt(pg_lambda2(5));
        for (int b = 0; b < (1 << d); ++b) {
            for (int i = 0; i < d; ++i) U[(size_t)p * d + i] = ((b >> i) & 1) ? -l : l;
            cls[p++] = 5;
        }
    }
    return p == n ? 0 : 1;
}

/* The five rule values (R7, R5, R3a, R3b, R1, scaled to the region) of one region. */
int orc_pagani_rules(int id, int d, const double *par, const double *lo, const double *len, double *Rout)
{
    const int n = orc_gm_count(d);
    if (!n) return 2;
    double *U = malloc(sizeof(double) * (size_t)n * d);
    int *cls = malloc(sizeof(int) * (size_t)n);
    if (!U || !cls || orc_gm_points(d, U, cls)) {
        free(U);
        free(cls);
        return 1;
    }
    double x[PG_DMAX], S[5] = {0, 0, 0, 0, 0}, vol = 1.0, W[25];
    for (int i = 0; i < d; ++i) vol *= len[i];
    for (int p = 0; p < n; ++p) {
        for (int i = 0; i < d; ++i) x[i] = lo[i] + 0.5 * len[i] * (1.0 + U[(size_t)p * d + i]);
        S[cls[p] - 1] += orc_integrand(id, d, par, x, 0);
    }
    orc_gm_rules(d, W);
    for (int r = 0; r < 5; ++r) {
        Rout[r] = 0.0;
        for (int k = 0; k < 5; ++k) Rout[r] += W[r * 5 + k] * S[k];
        Rout[r] *= vol / ldexp(1.0, d);
    }
    free(U);
    free(cls);
    return 0;
}

/* One region: I (degree-7 estimate), E (from the five rules), the split axis, and (if fourth != NULL) the
 * d fourth divided differences. Class sums are plain sequential sums in point order. */
int orc_pagani_evaluate(int id, int d, const double *par, const double *lo, const double *len, double *I,
                        double *E, int *axis, double *fourth)
{
    const int n = orc_gm_count(d);
    if (!n) return 2;
    double *U = malloc(sizeof(double) * (size_t)n * d);
    int *cls = malloc(sizeof(int) * (size_t)n);
    double *fv = malloc(sizeof(double) * (size_t)n);
    if (!U || !cls || !fv || orc_gm_points(d, U, cls)) {
        free(U);
        free(cls);
        free(fv);
        return 1;
    }
    double x[PG_DMAX], S[5] = {0, 0, 0, 0, 0}, vol = 1.0;
    for (int i = 0; i < d; ++i) vol *= len[i];
    for (int p = 0; p < n; ++p) {
        for (int i = 0; i < d; ++i) x[i] = lo[i] + 0.5 * len[i] * (1.0 + U[(size_t)p * d + i]);
        fv[p] = orc_integrand(id, d, par, x, 0);
        S[cls[p] - 1] += fv[p];
    }
    double W[25], R[5] = {0, 0, 0, 0, 0};
    orc_gm_rules(d, W);
    const double scale = vol / ldexp(1.0, d);
    for (int r = 0; r < 5; ++r) {
        for (int k = 0; k < 5; ++k) R[r] += W[r * 5 + k] * S[k];
        R[r] *= scale;
    }
    *I = R[0];
    *E = orc_pagani_error(R);
    /* fourth differences: class-2 points of axis i at 1 + 2i (+), 2 + 2i (-); class 3 at 1 + 2d + 2i, ... */
    const double r = pg_lambda2(2) / pg_lambda2(3), f0 = fv[0];
    /* rounding noise of a fourth difference is a few ulps of the largest |f| it combines: below
     * 1e-12 of that, differences are ties */
    double fscale = fabs(f0);
    for (int p = 1; p < 1 + 4 * d; ++p) fscale = fmax(fscale, fabs(fv[p]));
    double best = -1.0;
    int bi = 0;
    for (int i = 0; i < d; ++i) {
        const double a2 = fv[1 + 2 * i] + fv[2 + 2 * i] - 2.0 * f0;
        const double a3 = fv[1 + 2 * d + 2 * i] + fv[2 + 2 * d + 2 * i] - 2.0 * f0;
        const double D = fabs(a2 - r * a3);
        if (fourth) fourth[i] = D;
        const double tie = 1e-12 * fmax(fmax(D, best), fscale);
        if (D > best + tie) {
            best = D;
            bi = i;
        } else if (fabs(D - best) <= tie && len[i] > len[bi]) {
            bi = i;
        }
    }
    *axis = bi;
    free(U);
    free(cls);
    free(fv);
    return 0;
}

/* Adaptive driver (reading; the paper describes only the kernel). The unit cube starts as
 * init_split^d equal regions. Each iteration evaluates every active region; with the running
 * totals I = I_done + sum I_r and E = E_done + sum E_r it stops once E <= rel_tol |I|. Otherwise a
 * region whose error is within its share of the budget, E_r <= rel_tol |I| V_r, is finished
 * (its I_r, E_r join I_done, E_done); every other region is halved along its split axis, the
 * lower half first, children in the parents' order. The run also stops when no region is active,
 * after max_iters iterations, or when the next set would exceed max_regions.
 * out: [0] I, [1] E, [2] regions evaluated in total, [3] iterations, [4] status (0 converged,
 * 1 iteration limit, 2 region limit), [5] active regions at the end. */
int orc_pagani_integrate(int id, int d, const double *par, double rel_tol, int max_iters, int64_t max_regions,
                         int init_split, double *out)
{
    if (d < 2 || d > PG_DMAX || init_split < 1 || max_iters < 1 || max_regions < 1 || !(rel_tol > 0.0)) return 1;
    int64_t na = 1;
    for (int i = 0; i < d; ++i) na *= init_split;
    if (na > max_regions) return 1;
    double *lo = malloc(sizeof(double) * (size_t)na * d), *len = malloc(sizeof(double) * (size_t)na * d);
    if (!lo || !len) return 1;
    for (int64_t r = 0; r < na; ++r) {
        int64_t t = r;
        for (int i = 0; i < d; ++i) {
            const int c = (int)(t % init_split);
            t /= init_split;
            lo[r * d + i] = (double)c / init_split;
            len[r * d + i] = 1.0 / init_split;
        }
    }
    double I_done = 0.0, E_done = 0.0, I_tot = 0.0, E_tot = 0.0, evaluated = 0.0;
    int status = 1, it = 0;
    while (it < max_iters) {
        ++it;
        double *Ir = malloc(sizeof(double) * (size_t)na), *Er = malloc(sizeof(double) * (size_t)na);
        int *ax = malloc(sizeof(int) * (size_t)na);
        double sI = 0.0, sE = 0.0;
        for (int64_t r = 0; r < na; ++r) {
            orc_pagani_evaluate(id, d, par, lo + r * d, len + r * d, &Ir[r], &Er[r], &ax[r], NULL);
            sI += Ir[r];
            sE += Er[r];
        }
        evaluated += (double)na;
        I_tot = I_done + sI;
        E_tot = E_done + sE;
        if (E_tot <= rel_tol * fabs(I_tot)) {
            status = 0;
            free(Ir); free(Er); free(ax);
            break;
        }
        int64_t keep = 0;
        for (int64_t r = 0; r < na; ++r) {
            double vol = 1.0;
            for (int i = 0; i < d; ++i) vol *= len[r * d + i];
            if (!(Er[r] <= rel_tol * fabs(I_tot) * vol)) ++keep;
        }
        if (2 * keep > max_regions) {
            status = 2;
            free(Ir); free(Er); free(ax);
            break;
        }
        double *lo2 = malloc(sizeof(double) * (size_t)(2 * keep + 1) * d);
        double *len2 = malloc(sizeof(double) * (size_t)(2 * keep + 1) * d);
        int64_t k = 0;
        for (int64_t r = 0; r < na; ++r) {
            double vol = 1.0;
            for (int i = 0; i < d; ++i) vol *= len[r * d + i];
            if (Er[r] <= rel_tol * fabs(I_tot) * vol) {
                I_done += Ir[r];
                E_done += Er[r];
                continue;
            }
            for (int h = 0; h < 2; ++h) {
                for (int i = 0; i < d; ++i) {
                    lo2[k * d + i] = lo[r * d + i];
                    len2[k * d + i] = len[r * d + i];
                }
                len2[k * d + ax[r]] *= 0.5;
                if (h) lo2[k * d + ax[r]] += len2[k * d + ax[r]];
                ++k;
            }
        }
        free(Ir); free(Er); free(ax);
        free(lo); free(len);
        lo = lo2;
        len = len2;
        na = k;
        if (na == 0) {
            I_tot = I_done;
            E_tot = E_done;
            status = E_tot <= rel_tol * fabs(I_tot) ? 0 : 1;
            break;
        }
    }
    free(lo);
    free(len);
    out[0] = I_tot;
    out[1] = E_tot;
    out[2] = evaluated;
    out[3] = (double)it;
    out[4] = (double)status;
    out[5] = (double)na;
    return 0;
}
