// Definitions shared by the coupling-flow kernels: the layer layout, the tensor-core fragment
// helpers and the piecewise-quadratic transform of one axis (neural importance sampling,
// Mueller et al. 2019, Sec. 4). The per-layer kernels and the fused sampling kernel both use
// them, so both run the same arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

namespace mcubes {
struct IntegrandParams;
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

// Backward of one axis of a coupling layer in the density direction, y = CDF(x) and log q(x).
// In: the raw MLP outputs of the axis, x, gy = dL/dy and glq = dL/dlog q. Returns dL/dx and hands
// dL/draw_k (k = 0..2K) to put(k, value): K width logits, then K+1 edge-value logits.
template <int K, typename Put>
__device__ __forceinline__ float pq_backward(const float *raw, float x, float gy, float glq, Put put)
{
    float W[K], V[K + 1];
    widths_values<K>(raw, W, V);
    float X = 0.f, E = 0.f;
    int b = 0;
#pragma unroll
    for (int k = 0; k < K - 1; ++k) {
        E += W[k];
        if (x >= E) {
            X = E;
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
    const float delta = fminf(fmaxf(x - X, 0.f), Wb);
    const float dV = Vb1 - Vb;
    const float q = Vb + delta * dV / Wb;
    const float iq = 1.0f / q;
    const float gx = gy * q + glq * dV / (Wb * q);
    // dL/dW_k and dL/dV_k through y and log q
    float GW[K], GV[K + 1];
    const float dlq_dWlt = -dV / (Wb * q);                       // k < b (through delta)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float gw = 0.f;
        if (k < b) gw = gy * (0.5f * (V[k] + V[k + 1]) - q) + glq * dlq_dWlt;
        if (k == b) gw = -gy * delta * delta * dV / (2.f * Wb * Wb) - glq * delta * dV / (Wb * Wb) * iq;
        GW[k] = gw;
    }
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        float gv = 0.f;
        if (k < b) gv += gy * 0.5f * W[k];
        if (k >= 1 && k <= b) gv += gy * 0.5f * W[k - 1];
        if (k == b) gv += gy * (delta - delta * delta / (2.f * Wb)) + glq * (1.f - delta / Wb) * iq;
        if (k == b + 1) gv += gy * delta * delta / (2.f * Wb) + glq * (delta / Wb) * iq;
        GV[k] = gv;
    }
    // through the normalisation of V: V_k = e_k / Z
    float S = 0.f;
#pragma unroll
    for (int k = 0; k <= K; ++k) S += GV[k] * V[k];
#pragma unroll
    for (int k = 0; k < K; ++k) GW[k] -= 0.5f * (V[k] + V[k + 1]) * S;
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        const float c = 0.5f * ((k >= 1 ? W[k - 1] : 0.f) + (k < K ? W[k] : 0.f));
        put(K + k, V[k] * (GV[k] - c * S));
    }
    // through the softmax of the widths
    float SW = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) SW += GW[k] * W[k];
#pragma unroll
    for (int k = 0; k < K; ++k) put(k, W[k] * (GW[k] - SW));
    return gx;
}

// Bias + ReLU of an m16n8 accumulator row block (H/8 tiles, C layout), packed as bf16 into the
// operand layout of the next GEMM (H/16 k-tiles): n-tiles 2kt and 2kt+1 form k-tile kt.
template <int H>
__device__ __forceinline__ void relu_to_operand(const float (&acc)[H / 8][4], const float *bias, uint32_t (&a)[H / 16][4])
{
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int kt = 0; kt < H / 16; ++kt) {
        const int c = 16 * kt + 2 * t;
        a[kt][0] = pack_bf16(fmaxf(acc[2 * kt][0] + bias[c], 0.f), fmaxf(acc[2 * kt][1] + bias[c + 1], 0.f));
        a[kt][1] = pack_bf16(fmaxf(acc[2 * kt][2] + bias[c], 0.f), fmaxf(acc[2 * kt][3] + bias[c + 1], 0.f));
        a[kt][2] = pack_bf16(fmaxf(acc[2 * kt + 1][0] + bias[c + 8], 0.f), fmaxf(acc[2 * kt + 1][1] + bias[c + 9], 0.f));
        a[kt][3] = pack_bf16(fmaxf(acc[2 * kt + 1][2] + bias[c + 8], 0.f), fmaxf(acc[2 * kt + 1][3] + bias[c + 9], 0.f));
    }
}

// The last GEMM of a layer for output slots jp and jp + 1 (when < nB): o = W3 r2 + b3 into the
// warp's two FP32 slot buffers (16 rows x SW, row stride SW + 1).
template <int H, int K>
__device__ __forceinline__ void gemm3_pair(const __nv_bfloat16 *W3, const float *b3, const uint32_t (&a3)[H / 16][4],
                                           int nB, int jp, float *ob)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, NT3 = SW / 8, OS = SW + 1, LDH = H + 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int j = jp + hh;
        if (j < nB) {   // warp-uniform
            float acc[NT3][4] = {};
#pragma unroll
            for (int kt = 0; kt < H / 16; ++kt)
#pragma unroll
                for (int nt = 0; nt < NT3; ++nt) {
                    const __nv_bfloat16 *bp = W3 + (j * SW + nt * 8 + g) * LDH + kt * 16 + 2 * t;
                    mma16816(acc[nt], a3[kt], ld32(bp), ld32(bp + 8));
                }
            float *o = ob + hh * 16 * OS;
#pragma unroll
            for (int nt = 0; nt < NT3; ++nt) {
                const int c = nt * 8 + 2 * t;
                o[g * OS + c] = acc[nt][0] + b3[j * SW + c];
                o[g * OS + c + 1] = acc[nt][1] + b3[j * SW + c + 1];
                o[(g + 8) * OS + c] = acc[nt][2] + b3[j * SW + c];
                o[(g + 8) * OS + c + 1] = acc[nt][3] + b3[j * SW + c + 1];
            }
        }
    }
}

// ------------------------------------------------------------------------------ fused kernels
// Shared by the fused sampler and the fused training kernels: 8 warps a block, every layer's
// weights in a bf16 "mirror" that already has the shared-memory layout the kernels read.
//   W1 [H][kK0 + 8], W2 [H][H + 8], W3 [round16(|B| SW)][H + 8] (slot j at rows j SW .. j SW + 2K;
//   padding rows and columns zero), then b1 [H], b2 [H], b3 [|B| SW] in FP32; SW = 2K+1 rounded
//   up to 8.
constexpr int kFWarps = 8, kFThreads = kFWarps * 32;
constexpr int kFMaxLayers = 16;
constexpr int kFusedUnsupported = -1;   // internal status: the shape does not fit a fused kernel


struct FusedLayer {
    int nA, nB;
    int A[kMaxAB], B[kMaxAB];
    uint32_t off, bytes;                 // the layer's block in the mirror (bytes, multiples of 16)
    uint32_t oW2, oW3, ob1, ob2, ob3;    // byte offsets inside the block (W1 at 0)
    uint32_t pW1, pb1, pW2, pb2, pW3, pb3;   // offsets of the FP32 master parameters (floats)
};

struct FusedFlow {
    int L, H, K, SW;                     // SW: output slot width 2K+1 rounded up to 8
    uint32_t max_bytes, total_bytes;
    FusedLayer lay[kFMaxLayers];
};

inline uint32_t al16(uint32_t b) { return (b + 15u) & ~15u; }

// Host: the mirror layout of a flow shape. Returns false when the shape needs more layers than
// the fused path takes.
inline bool fused_layout(const Shape &S, FusedFlow &F)
{
    if (S.L > kFMaxLayers) return false;
    std::memset(&F, 0, sizeof(F));
    F.L = S.L;
    F.H = S.H;
    F.K = S.K;
    F.SW = (2 * S.K + 1 + 7) & ~7;
    const uint32_t LD0 = kK0 + 8, LDH = (uint32_t)S.H + 8;
    long long pos = 0;
    uint32_t off = 0;
    for (int l = 0; l < S.L; ++l) {
        const LayerDesc D = describe(S, l, pos);
        FusedLayer &Y = F.lay[l];
        Y.nA = D.nA;
        Y.nB = D.nB;
        for (int i = 0; i < kMaxAB; ++i) {
            Y.A[i] = D.A[i];
            Y.B[i] = D.B[i];
        }
        Y.pW1 = (uint32_t)D.offW1;
        Y.pb1 = (uint32_t)D.offb1;
        Y.pW2 = (uint32_t)D.offW2;
        Y.pb2 = (uint32_t)D.offb2;
        Y.pW3 = (uint32_t)D.offW3;
        Y.pb3 = (uint32_t)D.offb3;
        uint32_t b = al16(2u * S.H * LD0);
        Y.oW2 = b;
        b = al16(b + 2u * S.H * LDH);
        Y.oW3 = b;
        b = al16(b + 2u * (uint32_t)round16(D.nB * F.SW) * LDH);   // rows padded to 16 with zeros
        Y.ob1 = b;
        b = al16(b + 4u * S.H);
        Y.ob2 = b;
        b = al16(b + 4u * S.H);
        Y.ob3 = b;
        b = al16(b + 4u * (uint32_t)(D.nB * F.SW));
        Y.bytes = b;
        Y.off = off;
        off += b;
        F.max_bytes = std::max(F.max_bytes, b);
    }
    F.total_bytes = off;
    return true;
}

// Writes the mirror of the FP32 parameters d_params (defined with the sampler).
int build_mirror(const FusedFlow &F, const float *d_params, unsigned char *mirror, cudaStream_t s);

// ------------------------------------------------------------------------------ tcgen05 sampler
// The tensor-core (tcgen05) form of the fused sampler (flow_tc.cu): weights in the K-major,
// unswizzled core-matrix layout per layer (W1 [H][16], W2 [H][H], W3 [N3][H] bf16 with
// N3 = |B| SW rounded up to 16, then b1, b2, b3 in FP32).
struct TcLayer {
    int nA, nB, N3;
    int A[kMaxAB], B[kMaxAB];
    uint32_t off, bytes;
    uint32_t oW2, oW3, ob1, ob2, ob3;
    uint32_t pW1, pb1, pW2, pb2, pW3, pb3;
};

struct TcFlow {
    int L, H, K, SW;
    uint32_t max_bytes, total_bytes;
    TcLayer lay[kFMaxLayers];
};

struct TcSample {   // one iteration's stratification and Philox stream
    uint32_t m, p, g, key0, key1, ctr2_hi, job;
    int d, fid;
};

// The mirror layout of a shape; false when the tcgen05 sampler does not take it (H > 128,
// an output GEMM wider than 256, more than 16 layers).
bool tc_layout(const Shape &S, TcFlow &F);
int build_tc_mirror(const TcFlow &F, const float *d_params, unsigned char *mirror, cudaStream_t s);
// Samples [i0, i0 + n): x, log q (optional) and w = (f / F) / q; *err is set when a bounded wait
// expired. kFusedUnsupported when the shape does not fit (then use the mma.sync sampler).
int launch_flow_sample_tc(const TcFlow &F, const unsigned char *mirror, const TcSample &S,
                          const IntegrandParams &ip, long long i0, long long n, float *x, float *lq,
                          float *w, int *err, cudaStream_t s);

// Scratch of the fused training step (carved from the flow workspace).
struct FusedTrainWork {
    float *hs;                // L x n x d: the input of every layer
    float *gA, *gB;           // n x d each: dL/dh, ping-pong
    float *gl;                // n: dL/dlog q
    float *part;              // part_rows x part_stride: per-block partial gradients of one layer
    long long part_stride;
    int part_rows;
    unsigned char *mirror;    // the bf16 weight mirror
    int *err;                 // set by a tcgen05 kernel whose bounded wait expired (the step is then invalid)
};
constexpr int kFusedPartRowsMax = 1024;
constexpr int kFusedBwdRows = kFWarps * 16;   // samples per backward block tile

// Loss and gradient through the fused training kernels (flow_train.cu); grad and loss accumulate.
// Returns kFusedUnsupported when the shape's kernels do not fit the device's shared memory.
int fused_grad(const FusedFlow &F, const float *params, long long n, int d, const float *x, const float *w, int kind,
               float *grad, float *loss, const FusedTrainWork &W, cudaStream_t s);

// The same on the tcgen05 training kernels (flow_train_tc.cu), for widths 64 and 128 whose output
// GEMM is at most 256 wide; its mirror (the tcgen05 layout) must fit mirror_bytes. Returns
// kFusedUnsupported for other shapes.
int tc_grad(const Shape &S, const float *params, long long n, const float *x, const float *w, int kind, float *grad,
            float *loss, const FusedTrainWork &W, size_t mirror_bytes, cudaStream_t s);

// grad[e] += sum over rows r < rows of part[r pstride + e], e < npl, in a fixed order.
int launch_reduce_part(const float *part, int rows, long long pstride, int npl, float *grad, cudaStream_t s);

// One coupling layer on the 16 rows R0..R0+15 of a block's shared row set hs (row stride HS), run
// by one warp. The three GEMMs of the MLP chain through registers (the accumulator layout of
// m16n8k16 is its operand layout); the last GEMM's output goes to the warp's buffer ob (two
// 16 x (SW+1) FP32 slots) two axes at a time, and lane (row, half) transforms one (row, axis)
// pair with pq_transform (mode 0: density, 1: sampling). Returns the summed log pdf of the
// lane's row (the same in both halves).
template <int H, int K>
__device__ __forceinline__ float layer_rows16(const FusedLayer &Y, const unsigned char *wbuf, float *hs, int HS, int R0,
                                              float *ob, int mode)
{
    constexpr int SW = (2 * K + 1 + 7) & ~7, OS = SW + 1, LD0 = kK0 + 8, LDH = H + 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, row = lane & 15, half = lane >> 4;
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(wbuf);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(wbuf + Y.oW2);
    const __nv_bfloat16 *W3 = reinterpret_cast<const __nv_bfloat16 *>(wbuf + Y.oW3);
    const float *b1 = reinterpret_cast<const float *>(wbuf + Y.ob1);
    const float *b2 = reinterpret_cast<const float *>(wbuf + Y.ob2);
    const float *b3 = reinterpret_cast<const float *>(wbuf + Y.ob3);
    const int xA0 = 2 * t < Y.nA ? Y.A[2 * t] : -1, xA1 = 2 * t + 1 < Y.nA ? Y.A[2 * t + 1] : -1;
    // GEMM 1 operand: the A axes of rows R0 + g and R0 + g + 8, columns >= |A| zero
    uint32_t a1[4];
    {
        const float *hA = hs + (R0 + g) * HS, *hB = hs + (R0 + g + 8) * HS;
        a1[0] = pack_bf16(xA0 >= 0 ? hA[xA0] : 0.f, xA1 >= 0 ? hA[xA1] : 0.f);
        a1[1] = pack_bf16(xA0 >= 0 ? hB[xA0] : 0.f, xA1 >= 0 ? hB[xA1] : 0.f);
        a1[2] = 0u;
        a1[3] = 0u;
    }
    uint32_t a2[H / 16][4];
    {
        float acc[H / 8][4] = {};
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
            const __nv_bfloat16 *bp = W1 + (nt * 8 + g) * LD0 + 2 * t;
            mma16816(acc[nt], a1, ld32(bp), ld32(bp + 8));
        }
        relu_to_operand<H>(acc, b1, a2);
    }
    uint32_t a3[H / 16][4];
    {
        float acc[H / 8][4] = {};
#pragma unroll
        for (int kt = 0; kt < H / 16; ++kt)
#pragma unroll
            for (int nt = 0; nt < H / 8; ++nt) {
                const __nv_bfloat16 *bp = W2 + (nt * 8 + g) * LDH + kt * 16 + 2 * t;
                mma16816(acc[nt], a2[kt], ld32(bp), ld32(bp + 8));
            }
        relu_to_operand<H>(acc, b2, a3);
    }
    float lq = 0.f;
    for (int jp = 0; jp < Y.nB; jp += 2) {
        gemm3_pair<H, K>(W3, b3, a3, Y.nB, jp, ob);
        __syncwarp();
        const int j = jp + half;
        if (j < Y.nB) {
            float *hv = hs + (R0 + row) * HS + Y.B[j];
            float out, q;
            pq_transform<K>(ob + half * 16 * OS + row * OS, *hv, mode, out, q);
            *hv = out;
            lq += __logf(q);
        }
        __syncwarp();
    }
    return lq + __shfl_xor_sync(0xffffffffu, lq, 16);
}

}  // namespace flow
}  // namespace mcubes
