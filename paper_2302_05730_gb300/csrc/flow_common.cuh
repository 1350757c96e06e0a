// Definitions shared by the coupling-flow kernels: the layer layout, the tensor-core fragment
// helpers and the piecewise-quadratic transform of one axis (neural importance sampling,
// Mueller et al. 2019, Sec. 4). The per-layer kernels and the fused sampling kernel both use
// them, so both run the same arithmetic.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

namespace mcubes {
namespace flow {

constexpr int kTileRows = 64;      // samples per CTA tile (4 warps x 16 rows)
constexpr int kMaxAB = 8;          // |A|, |B| <= 8 (d <= 16)
constexpr int kK0 = 16;            // padded input width of the first GEMM

struct LayerDesc {
    int nA, nB, nout, nout_p;      // nout_p: nout rounded up to 16
    int A[kMaxAB], B[kMaxAB];
    long long offW1, offb1, offW2, offb2, offW3, offb3;
};

struct Shape {
    int d, L, H, K;
};

__host__ __device__ inline int round16(int x) { return (x + 15) & ~15; }

// Host: describe layer l of the flow.
inline LayerDesc describe(const Shape &s, int l, long long &pos)
{
    LayerDesc D;
    std::memset(&D, 0, sizeof(D));
    const int h = s.d / 2;
    int a = 0, b = 0;
    const int kind = l % 4;
    for (int i = 0; i < s.d; ++i) {
        bool inA;
        if (kind == 0) inA = i < h;
        else if (kind == 1) inA = i >= h;
        else if (kind == 2) inA = (i % 2) == 0;
        else inA = (i % 2) == 1;
        if (inA) D.A[a++] = i;
        else D.B[b++] = i;
    }
    D.nA = a;
    D.nB = b;
    D.nout = b * (2 * s.K + 1);
    D.nout_p = round16(D.nout);
    D.offW1 = pos; pos += (long long)s.H * a;
    D.offb1 = pos; pos += s.H;
    D.offW2 = pos; pos += (long long)s.H * s.H;
    D.offb2 = pos; pos += s.H;
    D.offW3 = pos; pos += (long long)D.nout * s.H;
    D.offb3 = pos; pos += D.nout;
    return D;
}

inline long long param_count(const Shape &s)
{
    long long pos = 0;
    for (int l = 0; l < s.L; ++l) describe(s, l, pos);
    return pos;
}

inline bool shape_ok(const Shape &s)
{
    if (s.d < 2 || s.d > 16 || s.L < 1 || s.L > 32) return false;
    if (s.H != 32 && s.H != 64 && s.H != 128) return false;
    if (s.K != 4 && s.K != 8 && s.K != 16 && s.K != 32) return false;
    return true;
}

// ------------------------------------------------------------------------------ mma helpers
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Widths W (softmax of the first K raw values) and edge pdf values V (exp of the next K+1,
// normalised so the piecewise-linear pdf integrates to one).
template <int K>
__device__ __forceinline__ void widths_values(const float *raw, float (&W)[K], float (&V)[K + 1])
{
    float mw = raw[0];
#pragma unroll
    for (int k = 1; k < K; ++k) mw = fmaxf(mw, raw[k]);
    float sw = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        W[k] = __expf(raw[k] - mw);
        sw += W[k];
    }
    const float isw = 1.0f / sw;
#pragma unroll
    for (int k = 0; k < K; ++k) W[k] *= isw;
    float mv = raw[K];
#pragma unroll
    for (int k = 1; k <= K; ++k) mv = fmaxf(mv, raw[K + k]);
#pragma unroll
    for (int k = 0; k <= K; ++k) V[k] = __expf(raw[K + k] - mv);
    float Z = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) Z += 0.5f * (V[k] + V[k + 1]) * W[k];
    const float iZ = 1.0f / Z;
#pragma unroll
    for (int k = 0; k <= K; ++k) V[k] *= iZ;
}

// One axis of a coupling layer. mode 0: density direction, out = CDF(v); mode 1: sampling
// direction, out = CDF^-1(v). q is the pdf at the point in x space (the input in mode 0, the
// output in mode 1).
template <int K>
__device__ __forceinline__ void pq_transform(const float *raw, float v, int mode, float &out, float &q)
{
    float W[K], V[K + 1];
    widths_values<K>(raw, W, V);
    // bin b: the last interior edge (of x in the density direction, of the cumulative mass in
    // the sampling direction) that v reaches; X, Y: the bin's left edge and the mass below it
    float X = 0.f, Y = 0.f, E = 0.f, M = 0.f;
    int b = 0;
#pragma unroll
    for (int k = 0; k < K - 1; ++k) {
        E += W[k];
        M += 0.5f * (V[k] + V[k + 1]) * W[k];
        if (v >= (mode == 0 ? E : M)) {
            X = E;
            Y = M;
            b = k + 1;
        }
    }
    float Wb = W[0], Vb = V[0], Vb1 = V[1];
#pragma unroll
    for (int k = 1; k < K; ++k)
        if (b == k) {
            Wb = W[k];
            Vb = V[k];
            Vb1 = V[k + 1];
        }
    if (mode == 0) {
        const float delta = fminf(fmaxf(v - X, 0.f), Wb);
        out = Y + delta * Vb + delta * delta * (Vb1 - Vb) / (2.f * Wb);
        q = Vb + delta * (Vb1 - Vb) / Wb;
    } else {
        const float r = fmaxf(v - Y, 0.f);
        const float disc = fmaxf(Vb * Vb + 2.f * r * (Vb1 - Vb) / Wb, 0.f);
        float delta = 2.f * r / (Vb + sqrtf(disc));
        delta = fminf(delta, Wb);
        out = fminf(X + delta, 1.0f);
        q = Vb + delta * (Vb1 - Vb) / Wb;
    }
}

}  // namespace flow
}  // namespace mcubes
