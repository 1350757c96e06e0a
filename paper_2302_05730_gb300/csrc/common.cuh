// Device-side building blocks shared by the m-Cubes kernels: constants, the launch parameter
// block of the V-Sample kernel, and the counter-based Philox4x32-10 generator.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcubes {

constexpr int kNB = 500;     // VEGAS bins per axis (Algorithm 2: B[500 d], C[500 d])
constexpr int kDMax = 16;
constexpr int kMaxBlockThreads = 256;   // V-Sample block size limit (launch bounds)

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4-word counter, 2-word key, ten rounds
// of the Philox S-box. Round: multiply words 0 and 2 by the two published constants (full
// 64-bit products), exchange halves and xor the high halves with words 1, 3 and the key;
// the key is bumped by the two Weyl increments between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct Words4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                         uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return Words4{c0, c1, c2, c3};
}

// Philox4x32-10 over the sampler's counters (t, q, s_j = ctr2_hi | j, job), with the work that
// does not depend on the draw hoisted out. The result is bit-identical to philox4x32_10.
//   Round 0 maps (t, q, s_j, job) to (a_j ^ q, b_j, hi(M0 t) ^ job ^ key1, lo(M0 t)) with
//   a_j = hi(M1 s_j) ^ key0 and b_j = lo(M1 s_j): a_j and b_j are launch constants, and
//   words 2 and 3 are constant over a sub-cube's draws.
//   Round 1 then multiplies word 2 by M1: hi and lo of that product are per-sub-cube values
//   too, and b_j ^ key0_1 (kept as bk_j) is a launch constant.
// The round keys key0 + r W0 and key1 + r W1 are stored, so the kernels read them as operands.
// Per draw that leaves 17 of the 20 64-bit products and no key additions.
constexpr int kPhiloxPreWords = 8;   // draw words j per sample (FP64 path at d = 16)
struct PhiloxPre {
    uint32_t k0[10], k1[10];         // round keys
    uint32_t a[kPhiloxPreWords];     // hi(M1 (ctr2_hi | j)) ^ key0
    uint32_t bk[kPhiloxPreWords];    // lo(M1 (ctr2_hi | j)) ^ (key0 + W0)
    uint32_t c;                      // job ^ key1
};
struct PhiloxCube {
    uint32_t x3;    // lo(M0 t): word 3 after round 0
    uint32_t h;     // hi(M1 x2), x2 = hi(M0 t) ^ job ^ key1: enters word 0 after round 1
    uint32_t y1;    // lo(M1 x2): word 1 after round 1
};

__host__ __device__ __forceinline__ void philox_prepare(PhiloxPre &pp, uint32_t key0, uint32_t key1,
                                                        uint32_t ctr2_hi, uint32_t job)
{
    for (int r = 0; r < 10; ++r) {
        pp.k0[r] = key0 + (uint32_t)r * kPhiloxW0;
        pp.k1[r] = key1 + (uint32_t)r * kPhiloxW1;
    }
    for (int j = 0; j < kPhiloxPreWords; ++j) {
        const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)(ctr2_hi | (uint32_t)j);
        pp.a[j] = (uint32_t)(p1 >> 32) ^ pp.k0[0];
        pp.bk[j] = (uint32_t)p1 ^ pp.k0[1];
    }
    pp.c = job ^ pp.k1[0];
}


// The cube state of sub-cube t (rounds 0 and 1's products of t), given job ^ key1.
__host__ __device__ __forceinline__ PhiloxCube philox_cube_k(uint32_t t, uint32_t job_xor_key1)
{
    const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)t;
    const uint32_t x2 = (uint32_t)(p0 >> 32) ^ job_xor_key1;
    const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)x2;
    return PhiloxCube{(uint32_t)p0, (uint32_t)(p1 >> 32), (uint32_t)p1};
}
__host__ __device__ __forceinline__ PhiloxCube philox_cube(uint32_t t, const PhiloxPre &pp)
{
    return philox_cube_k(t, pp.c);
}

// Rounds 1-9 of a draw: x0 = a_j ^ q (word 0 after round 0), bk_j, the cube state, and the round
// keys k0r(r), k1r(r).
template <class K0, class K1>
__host__ __device__ __forceinline__ Words4 philox_rounds_1_9(uint32_t x0, uint32_t bk, const PhiloxCube &cb, K0 k0r,
                                                             K1 k1r)
{
    const uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)x0;
    uint32_t c0 = cb.h ^ bk;
    uint32_t c1 = cb.y1;
    uint32_t c2 = (uint32_t)(p0 >> 32) ^ cb.x3 ^ k1r(1);
    uint32_t c3 = (uint32_t)p0;
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t m0 = (uint64_t)kPhiloxM0 * (uint64_t)c0;
        const uint64_t m1 = (uint64_t)kPhiloxM1 * (uint64_t)c2;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0r(r);
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1r(r);
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
    }
    return Words4{c0, c1, c2, c3};
}

// Philox4x32-10 of counter (t, q, ctr2_hi | j, job) from the prepared constants and t's cube state.
__host__ __device__ __forceinline__ Words4 philox_draw(uint32_t q, int j, const PhiloxCube &cb, const PhiloxPre &pp)
{
    return philox_rounds_1_9(
        pp.a[j] ^ q, pp.bk[j], cb, [&](int r) { return pp.k0[r]; }, [&](int r) { return pp.k1[r]; });
}

// The same from values a kernel keeps in registers (the batched kernel, whose per-job parameters
// are not launch constants): a_j and bk_j from philox_draw_consts, and the key itself, the round
// keys formed as the rounds need them.
__host__ __device__ __forceinline__ void philox_draw_consts(uint32_t key0, uint32_t ctr2_hi, int j, uint32_t &a_j,
                                                            uint32_t &bk_j)
{
    const uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)(ctr2_hi | (uint32_t)j);
    a_j = (uint32_t)(p1 >> 32) ^ key0;
    bk_j = (uint32_t)p1 ^ (key0 + kPhiloxW0);
}
__host__ __device__ __forceinline__ Words4 philox_draw_k(uint32_t q, uint32_t a_j, uint32_t bk_j, const PhiloxCube &cb,
                                                         uint32_t key0, uint32_t key1)
{
    return philox_rounds_1_9(
        a_j ^ q, bk_j, cb, [=](int r) { return key0 + (uint32_t)r * kPhiloxW0; },
        [=](int r) { return key1 + (uint32_t)r * kPhiloxW1; });
}

// The FP32 layout's uniforms of axes 4j .. 4j + 3 for sample (t, q): the four words of Philox call
// (t, q, ctr2_hi | j, job), low 23 bits each, times 2^-23.
__device__ __forceinline__ void uniforms_f32x4(uint32_t t, uint32_t q, uint32_t ctr2_hi, uint32_t job, uint32_t k0,
                                               uint32_t k1, int j, float u[4])
{
    const Words4 r = philox4x32_10(t, q, ctr2_hi | (uint32_t)j, job, k0, k1);
    u[0] = (float)(r.x & 0x7FFFFFu) * 1.1920928955078125e-7f;
    u[1] = (float)(r.y & 0x7FFFFFu) * 1.1920928955078125e-7f;
    u[2] = (float)(r.z & 0x7FFFFFu) * 1.1920928955078125e-7f;
    u[3] = (float)(r.w & 0x7FFFFFu) * 1.1920928955078125e-7f;
}

// Bounds checks of bounds-checked builds (-DMCUBES_CHECKED=1). mc_check(chk, i, n, site) is true
// when 0 <= i < n; otherwise it counts the failure in chk[0], records the first as
// site << 48 | index in chk[1], and returns false so that the caller skips the access. In normal
// builds it is the constant true.
#ifndef MCUBES_CHECKED
#define MCUBES_CHECKED 0
#endif
__device__ __forceinline__ bool mc_check(unsigned long long *chk, long long i, long long n, unsigned site)
{
#if MCUBES_CHECKED
    if (i >= 0 && i < n) return true;
    if (chk != nullptr && atomicAdd(&chk[0], 1ull) == 0ull)
        chk[1] = ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull);
    return false;
#else
    (void)chk; (void)i; (void)n; (void)site;
    return true;
#endif
}

// Integrand parameters as the kernels consume them. The FP64 path reads a and u as given;
// the FP32 path reads pre-scaled single-precision forms prepared on the host (see
// integrands.cuh for what each family stores).
struct IntegrandParams {
    double a[kDMax];
    double u[kDMax];
    double b[kDMax];   // FP64 auxiliary per axis (product peak: 1 / a^2)
    float fa[kDMax];
    float fu[kDMax];
    float fb[kDMax];   // FP32 auxiliary per axis (discontinuous: min(u, 1))
    float fc;          // FP32 scalar (oscillatory: u_0 mod 1)
    int d;
    double m[kDMax * kDMax];   // rotated Gaussian: the quadratic form M (row-major)
    float fm[kDMax * kDMax];   // ... as log2(e) M in single precision
};

// Everything one V-Sample launch needs, passed by value.
struct VsampleParams {
    const double *grid;      // d x (kNB + 1)
    double *C;               // d x kNB, accumulated (adjust) -- may be null otherwise
    double *sums;            // [2]: sum_t I_t, sum_t V_t (accumulated)
    const double *prev;      // previous iteration's estimate (prev[0] * prev_scale = I) or null
    double prev_scale;
    double *probe;           // per-cube probe output or null
    uint32_t probe_mask;     // cube t is probed when (t & probe_mask) == 0
    uint32_t probe_shift;
    uint32_t perm_mul;       // odd multiplier, coprime with the launch's thread count
    int ih_vmax_exp;         // fixed-point histogram: contributions below 2^ih_vmax_exp units take the
                             // integer path (set per launch so no bin's 64-bit sum can overflow)
    int fix_shift;           // fast FP64 kernel: fraction bits of its fixed-point table sums
    uint32_t m;              // sub-cubes
    uint32_t p;              // samples per sub-cube
    uint32_t g;              // strata per axis
    uint32_t key0, key1;     // Philox key = seed
    uint32_t ctr2_hi;        // iteration << 16
    uint32_t job;            // counter word 3
    int adjust;
    double R;                // nd / g (FP64)
    float R32;               // (float)(nd / g)
    double ycap;             // largest double below nd
    float ycap32;            // largest float below nd
    double inv_p;            // 1 / p
    double inv_pp1;          // 1 / (p (p - 1))
    double fscale;           // FP32 path: f = fscale * (kernel's scaled integrand)
    double log_fscale;       // log(fscale), or 0
    unsigned long long *chk; // bounds-checked builds: [0] failed checks, [1] the first one (else null)
    PhiloxPre ph;            // philox_prepare(key0, key1, ctr2_hi, job), filled at launch
    IntegrandParams ip;
};

}  // namespace mcubes
