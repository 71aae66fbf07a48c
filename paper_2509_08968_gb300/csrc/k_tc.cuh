// k_tc.cuh -- thin inline-PTX wrappers for the sm_103a tensor-core pipeline: mbarriers, TMA
// tensor loads, tensor-memory (TMEM) allocation and loads, tcgen05.mma and its descriptors.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace npf {
namespace tc {

// Limits of every bounded wait: a poll count and a wall-clock budget (try_wait itself suspends
// for a while between polls, so the time limit is the one that normally ends a stuck wait).
constexpr long long kWaitLimit = 1ll << 26;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long wall_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete; gives up after kWaitNs (or kWaitLimit
// polls), records `code` in *err and returns false; returns false at once when another role of
// the kernel has recorded an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code)
{
    const unsigned long long t0 = wall_ns();
    for (long long it = 0; it < kWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 1023) == 1023) {
            if (*(volatile int*)err) return false;
            if (wall_ns() - t0 > kWaitNs) break;
        }
    }
    atomicCAS(err, 0, code);
    return false;
}

// Arrive once on `bar` (plain arrive, no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---------------------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
// 2-D tiled load of the box at (x = inner element coordinate, y = row) into shared memory;
// completion is signalled on `bar` as transaction bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 3-D and 4-D tiled loads (coordinates innermost first): every slice plane of an operand tile
// in one copy.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            int w, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------- TMEM
// Executed by one full warp. Writes the allocated base address to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
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

// 32 lanes x 32-bit, 4 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------- MMA
// 1 on one lane of the (converged) warp, 0 on the others.
__device__ __forceinline__ uint32_t elect_one()
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r));
    return r;
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulation. The whole issuing warp runs
// the call (its descriptor arithmetic stays warp-uniform) and the lane with `leader` != 0 issues
// the MMA. The shared-memory descriptors are given as 32-bit halves (low: start address and
// leading offset, high: stride offset, version, layout) and the accumulate flag is fixed, so that
// a loop of MMAs over one stage costs a 32-bit add per operand and the instruction.
// COL keeps the A operand in the tensor core's collector buffer across consecutive MMAs that read
// the same A tile: 1 fills it (reading A from shared memory), 2 reads it from the buffer, 3 reads
// it from the buffer and releases it; 0 reads A from shared memory only.
#define NPF_MMA(QUAL)                                                                           \
    asm volatile("{\n\t.reg .pred p, q;\n\t.reg .b64 da, db;\n\t"                              \
                 "mov.b64 da, {%1, %3};\n\t"                                                     \
                 "mov.b64 db, {%2, %3};\n\t"                                                     \
                 "setp.ne.b32 p, %5, 0;\n\t"                                                     \
                 "setp.ne.b32 q, %6, 0;\n\t"                                                     \
                 "@q tcgen05.mma.cta_group::1.kind::f16" QUAL " [%0], da, db, %4, p;\n\t}"         \
                 ::"r"(d_tmem), "r"(a_lo), "r"(b_lo), "r"(hi), "r"(idesc), "n"(ACC ? 1 : 0),     \
                 "r"(leader)                                                                    \
                 : "memory")
template <bool ACC, int COL>
__device__ __forceinline__ void mma_bf16_lohi(uint32_t leader, uint32_t d_tmem, uint32_t a_lo,
                                              uint32_t b_lo, uint32_t hi, uint32_t idesc)
{
    if constexpr (COL == 0) NPF_MMA("");
    else if constexpr (COL == 1) NPF_MMA(".collector::a::fill");
    else if constexpr (COL == 2) NPF_MMA(".collector::a::use");
    else NPF_MMA(".collector::a::lastuse");
}
#undef NPF_MMA
// Shared-memory matrix descriptor of a K-major operand stored with the 64-byte swizzle (rows of 32
// BF16 = 64 bytes, 8-row atoms of 512 bytes), as two 32-bit halves: start address >> 4 at bits
// 0-13, leading byte offset (unused for swizzled K-major, 1) at 16-29; stride byte offset =
// 512 >> 4 at bits 32-45, descriptor version 1 at 46-47, layout type SWIZZLE_64B = 4 at 61-63.
// The low half is the same for every swizzle width.
__device__ __forceinline__ uint32_t sdesc_sw64_lo(uint32_t saddr)
{
    return ((saddr & 0x3FFFF) >> 4) | (1u << 16);
}
constexpr uint32_t kSdescSw64Hi = (512u >> 4) | (1u << 14) | (4u << 29);
// The same for the 32-byte swizzle (rows of 16 BF16 = 32 bytes, 8-row atoms of 256 bytes): stride
// byte offset 256 >> 4, layout type SWIZZLE_32B = 6.
constexpr uint32_t kSdescSw32Hi = (256u >> 4) | (1u << 14) | (6u << 29);

// Arrive once on `bar` when every tcgen05.mma issued so far by the leader lane has completed
// (issued by the leader lane of the warp that issued them).
__device__ __forceinline__ void mma_commit(uint32_t leader, uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.b32 q, %1, 0;\n\t"
        "@q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
        ::"r"(smem_u32(bar)), "r"(leader)
        : "memory");
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

}  // namespace tc
}  // namespace npf
