// tma.cuh -- mbarrier and TMA (cp.async.bulk.tensor) helpers shared by the
// kernels that stage tiles through the tensor memory accelerator (internal).
// Every wait is bounded by the global timer so that a copy that never lands
// ends in an error status instead of a hung kernel.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace asift {

constexpr unsigned long long kTmaWaitNs = 4000000000ull;   // a wait gives up after 4 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One potentially blocking test of a phase: the thread may be suspended (not
// spinning) for up to kTmaSuspendNs until the phase completes.
constexpr uint32_t kTmaSuspendNs = 1000000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %3;\nselp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kTmaSuspendNs)
        : "memory");
    return done != 0;
}

// Waits for the phase of `bar` with the given parity.  Gives up when another
// thread of the CTA has aborted (abort_flag set), or after limit_ns: then it
// raises the abort flag and records ASIFT_ERR_TIMEOUT.  With abort_flag NULL
// only the time limit applies.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int32_t *status, unsigned long long limit_ns = kTmaWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (global_ns() - t0 > limit_ns) {
            if (abort_flag) *abort_flag = 1;
            set_status(status, ASIFT_ERR_TIMEOUT);
            return false;
        }
    }
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 2-D tiled TMA load of the map's box at element coordinates (x, y) into
// shared memory, completing on `bar`.  x * element size must be a multiple of
// 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace asift
