// Bulk asynchronous global -> shared copies completed on an mbarrier
// (sm_90 and later: cp.async.bulk with mbarrier::complete_tx), as inline PTX.
//
// Rules the callers keep: source and destination 16-byte aligned, sizes a
// multiple of 16 bytes; one thread arms the barrier with the total byte count
// (arrive.expect_tx) before or with its copies; waits are bounded in time so a
// copy that never lands turns into an error status instead of a hang.
#pragma once

#include <cstdint>

namespace ei {

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Makes initialised barriers visible to the async proxy (the bulk copies).
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// A plain arrival (no transaction bytes); release semantics for the thread's
// earlier accesses.
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One bounded try: the thread may be suspended until the phase completes or
// about `hint_ns` nanoseconds pass (a hint; the hardware may wake it earlier).
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity, unsigned hint_ns = 0)
{
    unsigned ok;
    if (hint_ns == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(hint_ns)
            : "memory");
    }
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete, for at most
// `limit_ns` nanoseconds of wall time; false if it did not.  The tries are also
// capped at 2^22 (each suspends for up to ~20 us), so the wait ends even if the
// global timer did not advance.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned i = 1; i < (1u << 22); ++i) {
        if (mbar_try_wait(bar, parity, 20000u)) return true;      // sleep up to ~20 us a try
        if ((i & 15u) == 0 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// Copy `bytes` from global `src` to shared `dst`; completion is counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              unsigned bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 16-byte asynchronous global -> shared copy (cp.async, L2 only); src_bytes < 16
// fills the rest with zeros (0: nothing is read).  Completion per thread through
// commit / wait groups.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Orders this thread's earlier generic-proxy shared-memory writes before later
// async-proxy (bulk copy) accesses to the same locations.
__device__ __forceinline__ void proxy_fence_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2^x, the PTX approximate base-2 exponential (relative error about 2^-22;
// results below the normal range flush to zero).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace ei
