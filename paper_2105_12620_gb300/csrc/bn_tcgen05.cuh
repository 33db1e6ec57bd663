// bn_tcgen05.cuh — inline-PTX wrappers for the fifth-generation tensor core of sm_103a:
// tensor-memory (TMEM) allocation, tcgen05.mma of kind f16 issued by one thread of one CTA,
// its commit to an mbarrier, loads from tensor memory, and the shared-memory descriptor of a
// K-major operand stored in the 128-byte swizzled layout.
//
// Operand layout (K-major, 128-byte swizzle): a tile of R rows x 64 f16 (128 bytes per row).
// Row r starts at (r / 8) * 1024 + (r % 8) * 128; its 16-byte piece j (f16 8j .. 8j + 7) is
// stored at piece position j ^ (r % 8).  The tile base is 1024-byte aligned.  The descriptor of
// the k-th 16-element slice points 32 k bytes past the base; the hardware applies the same XOR
// to the addresses it forms, so one stored tile serves all four slices.
#pragma once

#include <cstdint>

namespace bn {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of f16 element k (0..63) of row r in a swizzled tile
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t r, uint32_t k)
{
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((((k >> 3) ^ r) & 7u) << 4) + (k & 7u) * 2u;
}

// shared-memory descriptor of slice k16 (0..3) of a swizzled K-major tile at shared address base
__host__ __device__ __forceinline__ uint64_t sw128_desc(uint32_t base, int k16)
{
    const uint32_t start = base + (uint32_t)k16 * 32u;
    uint64_t d = (uint64_t)((start >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;            // leading-dimension offset: unused by this layout
    d |= (uint64_t)(1024u >> 4) << 32;  // stride between 8-row groups
    d |= (uint64_t)1u << 46;            // descriptor version of this architecture
    d |= (uint64_t)2u << 61;            // 128-byte swizzle
    return d;
}

// instruction descriptor of kind f16: A and B f16, both K-major, D f32, shape M x N
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---- tensor memory ------------------------------------------------------------------------
// whole warp: allocate ncols columns (a power of two, 32..512); the address lands in *dst
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory stores of this thread become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival on *bar once every tcgen05.mma this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}

// D += A . B^T over one stage of K = 64 (four slices of 16), A from tensor memory at columns
// a_tmem .. a_tmem + 31, B from the swizzled tile whose slice-0 descriptor is bdesc0: the four
// products are issued back to back from one block (the tensor core's issue queue is short, so
// any work between them leaves it idle).  Slice k of B starts 32 k bytes later, i.e. 2 k in the
// descriptor's start-address field (which does not overflow for shared addresses below 256 KB).
__device__ __forceinline__ void mma4_f16_ts_acc(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc0,
                                                uint32_t idesc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 b1, b2, b3;\n\t.reg .b32 a1, a2, a3;\n\t"
        "setp.ne.b32 p, 1, 0;\n\t"
        "add.s64 b1, %2, 2;\n\tadd.s64 b2, %2, 4;\n\tadd.s64 b3, %2, 6;\n\t"
        "add.s32 a1, %1, 8;\n\tadd.s32 a2, %1, 16;\n\tadd.s32 a3, %1, 24;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc0), "r"(idesc)
        : "memory");
}

// whole warp: 16 registers per thread into 16 consecutive columns of the warp's 32 lanes,
// waiting for the stores to complete
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}

// whole warp: zero 16 consecutive columns of the warp's 32 lanes, waiting for the stores
__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr), "r"(0u)
        : "memory");
}

// whole warp: 16 consecutive columns of the warp's 32 lanes, waiting for the load
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

}  // namespace tc
}  // namespace bn
