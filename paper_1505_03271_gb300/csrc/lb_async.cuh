// lb_async.cuh -- bulk asynchronous global -> shared copies completed on
// shared-memory mbarriers (sm_90 and later: cp.async.bulk,
// mbarrier.arrive.expect_tx, mbarrier.try_wait.parity), and a wait on them
// that gives up after a time limit instead of spinning for ever.
//
// Rules these helpers rely on (PTX ISA, cp.async.bulk): source and
// destination addresses 16-byte aligned, size a multiple of 16 bytes.  The
// callers check both on the host before they launch.
#pragma once

#include <cstdint>

namespace lbgb {
namespace async {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// One arrival (the producer's expect_tx) completes each phase.
__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the asynchronous proxy.
__device__ __forceinline__ void bar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once and add `bytes` to the transaction count of the current phase.
__device__ __forceinline__ void bar_arrive_expect(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One plain arrival (release: this thread's earlier accesses are ordered
// before whatever the barrier's waiters do next).
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// True once the phase of the given parity has completed (acquire: the
// copied bytes are then visible to the waiting thread).  The thread is
// suspended in hardware until the phase completes or about `hint_ns`
// nanoseconds pass, so waiting warps take no issue slots from working ones.
__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, unsigned parity, unsigned hint_ns) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase, at most `limit_ns` nanoseconds; false when it ran out.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
    constexpr unsigned kHintNs = 20000;
    if (bar_try_wait(bar, parity, kHintNs)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (bar_try_wait(bar, parity, kHintNs)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Orders this thread's earlier shared-memory accesses before later
// asynchronous-proxy writes to the same memory (a ring slot being refilled).
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copies `bytes` from global memory to this CTA's shared memory; the
// completion counts against the transaction count of `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace async
}  // namespace lbgb
