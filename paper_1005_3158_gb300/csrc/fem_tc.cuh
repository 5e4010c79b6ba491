// Fifth-generation tensor-core helpers (tcgen05, sm_100a family) for the
// surrogate's dense layers: BF16 operands in shared memory, FP32
// accumulators in tensor memory (TMEM), one elected thread issuing the MMAs.
//
// Operand layout ("core-matrix", K-major, no swizzle).  An operand of R rows
// and K columns (bf16, K a multiple of 16, R a multiple of 8) is stored as
// core matrices of 8 rows x 8 columns (128 bytes, each row 16 contiguous
// bytes); core matrix (r / 8, k / 8) sits at byte
//     ((r / 8) * (K / 8) + k / 8) * 128,
// so core matrices adjacent along K are 128 bytes apart (the descriptor's
// leading-dimension offset) and adjacent 8-row groups K * 16 bytes apart
// (its stride-dimension offset).  One MMA consumes K = 16 columns, i.e. two
// core matrices along K: the k-th MMA of a product starts 256 * k bytes in.
//
// D = A B^T: A is M x K (rows = output rows), B is N x K (rows = output
// columns), D is M x N in TMEM, row i in lane i, column j in column base + j
// (FP32).  Warp w of the CTA reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once

#include <cstdint>

#include "fem_device.cuh"

namespace fem {
namespace tc {

// byte offset of element (r, k) in a core-matrix operand with K columns
__host__ __device__ __forceinline__ uint32_t core_off(uint32_t r, uint32_t k, uint32_t K)
{
    return (((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}
__host__ __device__ __forceinline__ uint32_t core_bytes(uint32_t R, uint32_t K) { return R * K * 2; }

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K), stride-dimension byte offset
// (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t K)
{
    const uint64_t lbo = 128, sbo = (uint64_t)K * 16;
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both
// operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation by one whole warp: the base address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[saddr_a] B[saddr_b]^T over K columns, M x N, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint32_t sa, uint32_t sb, uint32_t K,
                                         uint32_t M, uint32_t N, bool accumulate)
{
    const uint32_t id = idesc_bf16(M, N);
    for (uint32_t k = 0; k < K / 16; k++) {
        const uint64_t da = sdesc(sa + 256 * k, K), db = sdesc(sb + 256 * k, K);
        const uint32_t acc = (accumulate || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(id), "r"(acc)
            : "memory");
    }
}
// The same with A in two segments along K: K1 columns at sa1 (an operand of
// K1 columns) followed by K2 columns at sa2 (an operand of K2 columns); B
// is one operand of K1 + K2 columns.
__device__ __forceinline__ void mma_bf16_2seg(uint32_t tmem_d, uint32_t sa1, uint32_t K1, uint32_t sa2,
                                              uint32_t K2, uint32_t sb, uint32_t KB, uint32_t M,
                                              uint32_t N)
{
    const uint32_t id = idesc_bf16(M, N);
    for (uint32_t k = 0; k < (K1 + K2) / 16; k++) {
        const bool first = k < K1 / 16;
        const uint64_t da = first ? sdesc(sa1 + 256 * k, K1) : sdesc(sa2 + 256 * (k - K1 / 16), K2);
        const uint64_t db = sdesc(sb + 256 * k, KB);
        const uint32_t acc = k > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(id), "r"(acc)
            : "memory");
    }
}
// Arrive once on the mbarrier when every MMA issued so far by this thread
// has completed.
__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
// TMEM address of (this warp's lane quarter, column col)
__device__ __forceinline__ uint32_t lane_addr(uint32_t tbase, uint32_t col)
{
    return tbase + (((threadIdx.x >> 5) & 3u) << 21) + col;   // lane field: bits 16.., 32 lanes per warp
}

}  // namespace tc
}  // namespace fem
