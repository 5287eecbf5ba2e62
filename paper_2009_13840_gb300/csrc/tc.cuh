// Fifth-generation tensor-core helpers (sm_103a): tcgen05.mma with BF16
// operands in shared memory and an FP32 accumulator in tensor memory (TMEM).
//
// Operands are staged by ordinary stores into the no-swizzle K-major layout of
// 8 x 16-byte core matrices: the core matrix holding rows 8q..8q+7 and
// columns 8p..8p+7 of an R x K tile starts at byte (q * K/8 + p) * 128, its row
// i at +16 i.  The shared-memory descriptor of such a tile therefore has a
// leading-dimension (K direction) byte offset of 128 and a stride-dimension
// (row direction) byte offset of K/8 * 128; one MMA of K = 16 reads two core
// matrices along K, so step s starts 256 s bytes further.  The accumulator of
// an M = 128 tile is TMEM lane i = row i, column j = column j (32-bit each);
// warp w of a 128-thread group reads lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace hho {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// element offset of (row, k) in the core-matrix layout of a tile with K columns
__device__ __forceinline__ int core_off(int row, int k, int K) {
    return ((row >> 3) * (K >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp;
// the base address is written to *s_addr (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* s_addr, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_addr)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's ordinary shared-memory stores visible to the tensor cores
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for the given phase parity of the barrier with at most `limit` polls
// (each poll may suspend the thread for a bounded time).  Returns false when
// the limit is reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.u32 %0, 1, 0, P;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    return done != 0;
}

// D[128 x N] (TMEM) = A[128 x K] * B[K x N], A and B^T staged as K-major core
// tiles; issued by one thread, completion signalled on the barrier
__device__ __forceinline__ void mma_tile(uint32_t tmem, const void* sA, const void* sB, int K, int N, uint64_t* bar) {
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
    const uint32_t id = idesc_bf16(128, N);
    for (int s = 0; s < (K >> 4); ++s) {
        const uint64_t da = sdesc(a0 + 256u * s, 128u, sbo);
        const uint64_t db = sdesc(b0 + 256u * s, 128u, sbo);
        const uint32_t acc = s > 0;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(id), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace hho
