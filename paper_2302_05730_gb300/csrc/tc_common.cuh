// tcgen05 building blocks shared by the coupling-flow kernels on the fifth-generation tensor
// cores (the fused sampler, flow_tc.cu, and the training step, flow_train_tc.cu): K-major and
// MN-major shared-memory descriptors for kind::f16 MMAs with FP32 accumulators in TMEM, the
// single-thread MMA issue and commit, bounded mbarrier waits, TMEM loads and bulk copies.
//
// Operand layouts (bf16, no swizzle) are built from 8 x 8 core matrices of 16-byte rows; a buffer
// of `rows` x `cols` elements stores element (r, c) at cm_off(r, c, cols): core matrices 128 bytes
// apart along c, groups of 8 rows (cols / 8) x 128 bytes apart. Such a buffer serves a GEMM either
// as a K-major operand (K = its columns; lbo = 128, sbo = (cols / 8) x 128) or, read the other way,
// as an MN-major operand (K = its rows, MN = its columns; lbo = (cols / 8) x 128 along K, sbo = 128
// between core matrices along MN, and the transpose bit of that operand set in the instruction
// descriptor). The MN-major reading was checked against a host GEMM on a single CTA before any
// kernel used it.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mcubes {
namespace flow {
namespace tc {

constexpr int kTcRows = 128;          // samples per CTA tile = TMEM lanes of an M = 128 accumulator
constexpr int kTcCols = 256;          // TMEM columns a CTA allocates
constexpr uint32_t kTcWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major core-matrix offset (bytes) of element (r, k) of an operand with Kd columns.
__host__ __device__ __forceinline__ uint32_t cm_off(int r, int k, int Kd)
{
    return (uint32_t)((r >> 3) * (Kd >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start, leading-dimension offset (K direction), stride offset
// (8-row groups), the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M = 128.
__host__ __device__ __forceinline__ uint32_t mma_idesc(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

// D[tmem] (+)= A[128 x Kd] B[N x Kd]^T, Kd a multiple of 16, issued by the calling thread.
__device__ __forceinline__ void mma_issue(uint32_t tmem, const unsigned char *A, const unsigned char *B, int Kd, int N)
{
    const uint32_t idesc = mma_idesc(N), sbo = (uint32_t)(Kd >> 3) * 128u;
    for (int kk = 0; kk < Kd / 16; ++kk) {
        const uint64_t ad = smem_desc(su32(A) + kk * 256, 128, sbo);
        const uint64_t bd = smem_desc(su32(B) + kk * 256, 128, sbo);
        const uint32_t acc = kk > 0 ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mbar)));
}

// Bounded wait for the mbarrier phase `parity`; false when it expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (uint32_t it = 0; it < kTcWaitLimit && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(su32(mbar)), "r"(parity));
    return done != 0;
}

// Eight FP32 columns [col, col + 8) of this warp's 32 TMEM lanes: v[j] = row's column col + j.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// One thread: expect `bytes` on mbar and start the bulk copy global -> shared that delivers them.
// src, dst and bytes are multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(mbar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(mbar))
                 : "memory");
}

__device__ __forceinline__ void before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;"); }

}  // namespace tc
}  // namespace flow
}  // namespace mcubes

namespace mcubes {
namespace flow {
namespace tc {

// One MMA operand: a rows x cols bf16 buffer in the core-matrix layout, read K-major (K = its
// columns) or MN-major (K = its rows), its MN extent starting at mn0 (a multiple of 8).
struct Opnd {
    const unsigned char *base;
    int cols;
    bool mn;
    int mn0;
};

// Descriptor of K-step kk (16 elements of K) of an operand.
__device__ __forceinline__ uint64_t opnd_desc(const Opnd &o, int kk)
{
    const uint32_t group = (uint32_t)(o.cols >> 3) * 128u;   // bytes between 8-row groups
    if (!o.mn) return smem_desc(su32(o.base) + (uint32_t)(o.mn0 >> 3) * group + (uint32_t)kk * 256u, 128u, group);
    return smem_desc(su32(o.base) + (uint32_t)kk * 2u * group + (uint32_t)(o.mn0 >> 3) * 128u, group, 128u);
}

// D[tmem] (+)= A B^T with M = 128 rows of A, N rows of B and Kd (a multiple of 16) along K, from
// operands read K-major or MN-major; accumulate adds to D, else the first K-step overwrites it.
// Issued by the calling thread.
__device__ __forceinline__ void mma_ab(uint32_t tmem, const Opnd &A, const Opnd &B, int Kd, int N, bool accumulate)
{
    const uint32_t idesc = mma_idesc(N) | (A.mn ? (1u << 15) : 0u) | (B.mn ? (1u << 16) : 0u);
    for (int kk = 0; kk < Kd / 16; ++kk) {
        const uint64_t ad = opnd_desc(A, kk), bd = opnd_desc(B, kk);
        const uint32_t acc = (kk > 0 || accumulate) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

}  // namespace tc
}  // namespace flow
}  // namespace mcubes
