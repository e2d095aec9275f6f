// lcq_pipe.cuh -- shared-memory staging for the streaming kernels: 1-D bulk
// asynchronous copies (cp.async.bulk, the TMA engine) from global memory into
// shared memory, completion tracked by mbarriers with transaction counts.
// Every wait is bounded so that a kernel can always return.
#pragma once

#include <cstdint>

namespace lcq {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive once and announce `bytes` of incoming transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Global -> shared bulk copy; bytes and both addresses multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Invariant: no bulk copy is outstanding when a CTA leaves the kernel; a copy
// still in flight would land in shared memory that the SM may already have
// handed to another CTA.  Thread 0, the only thread that issues copies into a
// ring of STAGES stage buffers, calls this on every way out of its loop (also
// after a timeout or an abort): `filled` stages were issued, the last STAGES
// of them sit in distinct slots (older ones were consumed before their slot
// was refilled), and armed(f) says whether stage f was armed (an arrive, with
// or without a copy).  Waiting on a phase that has already completed returns
// at once, so consumed stages cost one poll each.  Returns false if a wait
// gave up (the copy engine never finished; the caller records an error).
template <int STAGES, typename Armed>
__device__ __forceinline__ bool drain_stages(uint64_t* bars, uint32_t filled, Armed&& armed, uint32_t limit) {
    const uint32_t lo = filled > (uint32_t)STAGES ? filled - (uint32_t)STAGES : 0u;
    bool ok = true;
    for (uint32_t f = lo; f < filled; f++)
        if (armed(f) && !mbar_wait(&bars[f % STAGES], (f / STAGES) & 1u, limit)) ok = false;
    return ok;
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy writes (a buffer is refilled after it was read).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace lcq

namespace lcq {

// Named barrier over the first `nthreads` threads of the CTA (the compute
// warps of a warp-specialised kernel); id 0 is reserved for __syncthreads.
__device__ __forceinline__ void named_barrier_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Bounded wait that also gives up when another thread of the CTA raised the
// abort flag (so that every warp leaves the kernel after one timeout).
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, uint32_t limit,
                                                   volatile uint32_t* abort_flag) {
    for (uint32_t i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 63u && *abort_flag) return false;
    }
    return false;
}

}  // namespace lcq

namespace lcq {

// Named barrier that also ORs a predicate over its participants: every
// participant gets the same answer, so a decision taken from it (such as
// leaving the loop after a timeout) is uniform and no thread is left waiting
// at a later barrier.
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

}  // namespace lcq
