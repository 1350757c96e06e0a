// Bit-level FP64 steps of the fast FP64 V-Sample kernel (vsample64.cuh; paper Sec. 3.2, Algorithm 2),
// usable on the host as well as on the device, so that they can be checked on the CPU against IEEE
// FP64 arithmetic:
//   - yn = fl(fl(c + u) R) with integer operations, rounded as the two FP64 operations round;
//   - the bin k = floor(yn) and the offset's bits from yn's bits;
//   - the FP32-found integer of an argument reduction, and small integers as FP64 values;
//   - 2^E exp(x) and cos(2 pi t) from per-block tables and their reduced arguments' series.
// On the device each step is the CUDA intrinsic it names; on the host, portable C++ with the same
// rounding (IEEE round to nearest even; a host build must not contract a * b + c).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include <vector_types.h>

#if defined(__CUDACC__)
#define MC_BITS_FN __host__ __device__ __forceinline__
#else
#define MC_BITS_FN inline
#endif

namespace mcubes {

constexpr int kExpTab = 256;     // 2^(j / 256), j = 0..255
constexpr int kCosTab = 256;     // cos and sin of 2 pi j / 256

// ln 2 / 256 in two parts: the high part has 34 significant bits, so k * hi is exact for |k| < 2^19.
constexpr double kLn2by256Hi = 0x1.62e42fef80000p-9;
constexpr double kLn2by256Lo = 0x1.1cf79abc9e3b4p-44;
constexpr float k256byLn2f = 369.32993f;
constexpr double kTwoPi64 = 0x1.921fb54442d18p+2;
constexpr double kRoundMagic = 0x1.8p52;   // 1.5 2^52: adding it rounds to an integer in the low word
constexpr float kRoundMagicF = 12582912.0f;   // 1.5 2^23, the same in FP32

namespace bits {

MC_BITS_FN int clz32(unsigned x)
{
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return x != 0u ? __builtin_clz(x) : 32;
#endif
}

MC_BITS_FN int clz64(unsigned long long x)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x != 0ull ? __builtin_clzll(x) : 64;
#endif
}

MC_BITS_FN unsigned long long umulhi64(unsigned long long a, unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

MC_BITS_FN unsigned long long dbits(double x)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

MC_BITS_FN double from_dbits(unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

MC_BITS_FN int hi(double x)
{
#ifdef __CUDA_ARCH__
    return __double2hiint(x);
#else
    return (int)(uint32_t)(dbits(x) >> 32);
#endif
}

MC_BITS_FN int lo(double x)
{
#ifdef __CUDA_ARCH__
    return __double2loint(x);
#else
    return (int)(uint32_t)dbits(x);
#endif
}

MC_BITS_FN double hilo(int h, int l)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double(h, l);
#else
    return from_dbits(((unsigned long long)(uint32_t)h << 32) | (uint32_t)l);
#endif
}

MC_BITS_FN float from_fbits(int b)
{
#ifdef __CUDA_ARCH__
    return __int_as_float(b);
#else
    float x;
    std::memcpy(&x, &b, sizeof x);
    return x;
#endif
}

MC_BITS_FN int fbits(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_int(x);
#else
    int b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

MC_BITS_FN float fadd_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}

MC_BITS_FN float fmul_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

MC_BITS_FN double fma_rn(double a, double b, double c)
{
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

MC_BITS_FN double exp_lib(double x)
{
#ifdef __CUDA_ARCH__
    return exp(x);
#else
    return std::exp(x);
#endif
}

MC_BITS_FN double ldexp_lib(double x, int e)
{
#ifdef __CUDA_ARCH__
    return ldexp(x, e);
#else
    return std::ldexp(x, e);
#endif
}

}  // namespace bits

// The bits of yn = fl(fl(c + u) R) (both FP64 roundings, to nearest even) for integers 0 <= c < 2^11 and
// u = bits 2^-52 (bits < 2^52), from hi = c 2^20 + (bits >> 32) and lo = the low 32 bits, with integer
// operations only. N = c 2^52 + bits has bit length L; fl(c + u) = q 2^(L - 105), q = N cut to 53 bits
// and rounded to nearest even (exact when L <= 53); R = Rm 2^(eR - 52) (Rm with its leading bit); yn's
// significand is the 105- or 106-bit product q Rm cut to 53 bits and rounded to nearest even. 0 for
// c + u = 0.
MC_BITS_FN unsigned long long cu_times_r_bits(uint32_t hi, uint32_t lo, unsigned long long Rm, int eR)
{
    const unsigned long long N = ((unsigned long long)hi << 32) | lo;
    int L = 64 - bits::clz64(N);
    unsigned long long q;
    if (L > 53) {
        const int s = L - 53;
        q = (N + (1ull << (s - 1)) - 1ull + ((N >> s) & 1ull)) >> s;
        if (q >> 53) {   // rounded up to 2^53
            q >>= 1;
            ++L;
        }
    } else {
        q = N << (53 - L);
    }
    const unsigned long long plo = q * Rm;
    const unsigned long long phi = bits::umulhi64(q, Rm);   // q Rm < 2^106: phi < 2^42
    const int sh = 52 + (int)(phi >> 41);                   // bits below the 53-bit significand
    unsigned long long sig = (phi << (64 - sh)) | (plo >> sh);
    const unsigned long long rem = plo & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    sig += (rem > half || (rem == half && (sig & 1ull))) ? 1ull : 0ull;
    // yn = sig 2^(E - 52) with E = L - 105 + eR + sh; sig = 2^53 carries into the exponent field
    const int E = L - 105 + eR + sh;
    return N != 0ull ? ((unsigned long long)(E + 1022) << 52) + sig : 0ull;
}

// Bin and offset of 0 <= yn < 512 from its bits (integer operations only): k = floor(yn), and
// the bits of G = 1 + (yn - k) (exact for yn >= 1; for yn < 1, 1 + yn cut to 52 fraction bits).
MC_BITS_FN int split_bin(unsigned long long yb, unsigned long long &gbits)
{
    const int e = (int)(yb >> 52) - 1023;                          // yn >= 0
    const unsigned long long mant = yb & 0x000FFFFFFFFFFFFFull;
    const unsigned long long M = mant | 0x0010000000000000ull;
    unsigned long long frac;
    int k;
    if (e >= 0) {
        frac = (mant << e) & 0x000FFFFFFFFFFFFFull;
        k = (int)(M >> (52 - e));
    } else {
        const int sh = -e < 63 ? -e : 63;
        frac = M >> sh;
        k = 0;
    }
    gbits = 0x3FF0000000000000ull | frac;
    return k;
}

// x cut to 24 significant bits, as an FP32 value (0 below 2^-126); |x| < 2^128.
MC_BITS_FN float f32_cut(double x)
{
    const int hx = bits::hi(x);
    const int ex = (hx >> 20) & 0x7FF;
    const int b = (hx & (int)0x80000000) | ((ex - 896) << 23) | ((hx & 0xFFFFF) << 3) |
                  (int)((unsigned)bits::lo(x) >> 29);
    return ex > 896 ? bits::from_fbits(b) : 0.0f;
}

// The nearest integer to v (|v| < 2^22) in FP32: adding 1.5 2^23 rounds it into the low bits.
MC_BITS_FN int f32_round_int(float v)
{
    return bits::fbits(bits::fadd_rn(v, kRoundMagicF)) - 0x4B400000;
}

// k as an FP64 value (|k| <= 2^20) from its bits with integer operations: the sign, the exponent
// of the leading one and the bits below it as the top fraction bits.
MC_BITS_FN double small_int_to_double(int k)
{
    const unsigned a = (unsigned)(k < 0 ? -k : k);
    const int e = a != 0u ? 31 - bits::clz32(a) : 0;   // a in [2^e, 2^(e+1)), e <= 20
    const int h = (k < 0 ? (int)0x80000000 : 0) | ((1023 + e) << 20) | (int)((a ^ (1u << e)) << (20 - e));
    return a != 0u ? bits::hilo(h, 0) : 0.0;
}

// 2^E exp(x): x = (256 m + j) ln2/256 + r with |r| <= 0.56 ln2/256 (k = 256 m + j within one of the
// nearest integer to x 256/ln2), so 2^E exp(x) = 2^(m + E) 2^(j/256) e^r; e^r - 1 from its Taylor
// series through r^4 (remainder below 7e-17), 2^(j/256) from the block's table T, m + E added to the
// exponent field. 7 FP64 operations. Outside |x| < 708, or where the result leaves the normal
// range, the library's exp and ldexp.
MC_BITS_FN double exp_tab(double x, int E, const double *T)
{
    if ((bits::hi(x) & 0x7FFFFFFF) >= 0x40862000) return bits::ldexp_lib(bits::exp_lib(x), E);   // |x| >= 708
    const int k = f32_round_int(bits::fmul_rn(f32_cut(x), k256byLn2f));
    const double kf = small_int_to_double(k);
    double r = bits::fma_rn(kf, -kLn2by256Hi, x);
    r = bits::fma_rn(kf, -kLn2by256Lo, r);
    double q = bits::fma_rn(r, 1.0 / 24.0, 1.0 / 6.0);
    q = bits::fma_rn(q, r, 0.5);
    q = bits::fma_rn(q, r, 1.0);
    q = q * r;                                   // e^r - 1
    const double tj = T[k & (kExpTab - 1)];
    const double y = bits::fma_rn(tj, q, tj);    // 2^(j/256) e^r, in [0.99, 2.01)
    const int m = (k >> 8) + E;
    const int hy = bits::hi(y);
    const int ey = ((hy >> 20) & 0x7FF) + m;
    if (ey <= 0 || ey >= 0x7FF) return bits::ldexp_lib(y, m);
    return bits::hilo(hy + (m << 20), bits::lo(y));
}

// cos(2 pi t) for |t| < 2^40 turns: t = k/256 + r, |r| <= 0.63/256 (k within one of the nearest
// integer to 256 t: found in FP32 for |t| < 2^12, else rounded in FP64), r exact; theta = 2 pi r and
// cos(2 pi t) = C_j cos(theta) - S_j sin(theta), j = k mod 256; cos(theta) - 1 through theta^6 and
// sin(theta) through theta^5 (remainders below 5e-17). 11 FP64 operations below 2^12 turns.
// CS holds (C_j, S_j) pairs.
MC_BITS_FN double cos_turns(double t, const double2 *CS)
{
    int k;
    double kf;
    if ((bits::hi(t) & 0x7FFFFFFF) < 0x40B00000) {   // |t| < 2^12
        k = f32_round_int(bits::fmul_rn(f32_cut(t), 256.0f));
        kf = small_int_to_double(k);
    } else {
        const double kd = bits::fma_rn(t, 256.0, kRoundMagic);
        k = bits::lo(kd);
        kf = kd - kRoundMagic;
    }
    const double r = bits::fma_rn(kf, -1.0 / 256.0, t);
    const double th = r * kTwoPi64;
    const double z = th * th;
    double c = bits::fma_rn(z, -1.0 / 720.0, 1.0 / 24.0);
    c = bits::fma_rn(c, z, -0.5);
    c = c * z;                                   // cos(theta) - 1
    double s = bits::fma_rn(z, 1.0 / 120.0, -1.0 / 6.0);
    s = s * z;
    s = bits::fma_rn(th, s, th);                 // sin(theta)
    const double2 cs = CS[k & (kCosTab - 1)];
    return bits::fma_rn(-cs.y, s, bits::fma_rn(cs.x, c, cs.x));
}

}  // namespace mcubes
