// mbarrier and bulk-copy (TMA) helpers shared by the kernels: an mbarrier in
// shared memory, bounded waits on its phases, and the one-dimensional bulk copy
// from global to shared memory that completes on an mbarrier (the copy engine
// moves the bytes; the issuing thread only posts one instruction).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "ft_internal.cuh"

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of phase `parity`: false once `limit` SM
// cycles have passed (FT_WAIT_CYCLES, about 2 s, by default).  The limit is
// checked before every try, so a limit of 0 gives up at once (the plan's test
// setting that exercises the timeout path).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = FT_WAIT_CYCLES) {
    const long long t0 = clock64();
    for (;;) {
        if (clock64() - t0 >= limit) return false;
        if (mbar_try(mbar, parity)) return true;
    }
}
// the calling thread's arrival, announcing `bytes` of bulk copies to come
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global to this block's shared memory, completing on mbar
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(mbar)
        : "memory");
}

// prefetch into L2 of the box at (x, y, z) of the tensor *tmap (a hint: no
// shared memory, nothing to wait for; coordinates outside the tensor fetch nothing)
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* tmap, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// 3-D tiled tensor copy (TMA) of the box at (x, y, z) of the tensor described by
// *tmap (a __grid_constant__ kernel parameter) into this block's shared memory,
// completing on mbar; x times the element size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* tmap, int x, int y, int z,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}
