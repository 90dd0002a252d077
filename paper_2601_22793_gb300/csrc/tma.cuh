// Tensor-memory-accelerator (TMA) bulk copies and mbarrier completion, as
// inline PTX for sm_90 and later.  A 2-D tiled copy moves a box of a tensor
// described by a CUtensorMap (built on the host) between global and shared
// memory without passing through the registers or the L1 cache of the SM.
// Loads signal an mbarrier with the bytes they deliver; stores are tracked as
// bulk groups of the issuing thread.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace epr_tma {

__device__ __forceinline__ unsigned int smem_u32(const void* p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// arrive once and announce `bytes` of transactions still to complete
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// wait for the phase with the given parity to complete; gives up after
// `limit` polls (each poll may suspend the thread for a short while) and
// returns false
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned int parity, unsigned int limit)
{
    const unsigned int a = smem_u32(bar);
    for (unsigned int i = 0; i < limit; ++i) {
        unsigned int ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// make this thread's generic-proxy shared-memory writes visible to later
// bulk (async-proxy) operations
__device__ __forceinline__ void fence_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// order generic-proxy global accesses before later async-proxy ones
__device__ __forceinline__ void fence_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// box at element coordinates (x, y) of the map -> shared memory at dst
__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                        uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared memory at src -> box at element coordinates (x, y) of the map
__device__ __forceinline__ void store_2d(const CUtensorMap* map, int x, int y, const void* src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// wait until every committed bulk group of this thread has finished reading
// its shared-memory source (the writes complete on their own; the end of the
// grid makes them visible to later grids)
__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

}  // namespace epr_tma
