// Device-side building blocks shared by the drain, payload and setup kernels:
// scoped loads/stores, bounded waits, and a bounded multi-producer /
// multi-consumer queue of 32-bit values.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "layout.h"

namespace cafgpu {

// ---------------------------------------------------------------------------
// Scoped memory operations.  ".gpu" orders accesses between warps of this
// GPU; ".sys" additionally orders them with the host (pinned memory that the
// host polls or writes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_acquire_gpu(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t *p, uint32_t v) {
    asm volatile("st.release.sys.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(uint64_t *p, uint64_t v) {
    asm volatile("st.release.sys.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.sys.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Acquire-release compare-and-swap of a 32-bit word (gpu scope): the
// actor-state handshake between a claim that parks an actor (a release store
// of WAITING) and a producer that wakes or claims it, so the head the claim
// published is visible to whoever claims the actor next.
__device__ __forceinline__ uint32_t cas_acq_rel_gpu(uint32_t *p, uint32_t expect, uint32_t desired) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "l"(p), "r"(expect), "r"(desired)
                 : "memory");
    return old;
}
__device__ __forceinline__ uint32_t cas_u32(uint32_t *p, uint32_t expect, uint32_t desired) {
    return atomicCAS(reinterpret_cast<unsigned int *>(p), expect, desired);
}
__device__ __forceinline__ uint64_t cas_u64(uint64_t *p, uint64_t expect, uint64_t desired) {
    return atomicCAS(reinterpret_cast<unsigned long long *>(p), (unsigned long long)expect,
                     (unsigned long long)desired);
}
__device__ __forceinline__ uint64_t add_u64(uint64_t *p, uint64_t v) {
    return atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}
__device__ __forceinline__ uint32_t add_u32(uint32_t *p, uint32_t v) {
    return atomicAdd(reinterpret_cast<unsigned int *>(p), v);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// ---------------------------------------------------------------------------
// Shared-memory barriers and bulk asynchronous copies (TMA engine, sm_90+).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t saddr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr) : "memory");
    return v;
}
// Shared load at a register address plus a constant byte offset (folded into
// the instruction).
template <uint32_t kOff>
__device__ __forceinline__ uint32_t lds_u32_at(uint32_t saddr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(saddr), "n"(kOff) : "memory");
    return v;
}
// Make barrier initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's generic-proxy shared-memory accesses before later
// asynchronous-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
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
// Bulk copy `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Bounded waits.  Every spin in the device code goes through WaitClock: it
// gives up after `limit_ns` of %globaltimer time, after which the caller
// records an error code in the control block and unwinds.
// ---------------------------------------------------------------------------
struct WaitClock {
    uint64_t deadline;
    uint32_t spins;
    __device__ __forceinline__ explicit WaitClock(uint64_t limit_ns)
        : deadline(globaltimer() + limit_ns), spins(0) {}
    // Back off briefly; false once the deadline has passed.
    __device__ __forceinline__ bool again() {
        ++spins;
        if (spins > 8) __nanosleep(spins < 64 ? 32 : 256);
        return (spins & 15u) != 0 || globaltimer() < deadline;
    }
};

__device__ __forceinline__ void raise_error(DevCtl *ctl, uint32_t code, uint32_t site) {
    atomicCAS(reinterpret_cast<unsigned int *>(&ctl->error_word), 0u, code | (site << 8));
}

// ---------------------------------------------------------------------------
// Bounded MPMC queue: an array of cells with sequence numbers, positions
// handed out by atomic adds on the tail (push) and head (pop) -- no CAS retry
// loop, so many CTAs can pop at once without the pops serialising on one
// word, and each pop is served in the order it arrived.
//
// A pop first reserves an item on `avail` (published items not yet reserved;
// an add of -1 that finds it <= 0 is undone and the pop reports empty), then
// takes the next head position.  Reservations never exceed the items
// published, so every position a pop takes is (or is about to be) filled by a
// push that already holds it; the pop waits, bounded, for that cell.  A push
// takes a tail position, waits (bounded) until the cell's previous occupant
// has been popped, publishes the value and then counts it in `avail`.  Each
// value is in the queue at most once per push; capacity is a power of two and
// is sized by the host so that a push never needs to wait for space.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t q_avail(QueueHdr *q) {
    return (int64_t)ld_relaxed_gpu(reinterpret_cast<const uint64_t *>(&q->avail));
}
__device__ __forceinline__ int64_t q_avail_add(QueueHdr *q, int64_t v) {
    return (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&q->avail), (unsigned long long)v);
}

__device__ __forceinline__ bool q_push(QueueHdr *q, QCell *cells, uint32_t v, uint64_t limit_ns) {
    uint64_t pos = add_u64(&q->enq, 1);
    QCell *c = &cells[pos & q->mask];
    if (ld_acquire_gpu(&c->seq) != pos) {
        WaitClock w(limit_ns);
        while (ld_acquire_gpu(&c->seq) != pos) {
            if (!w.again()) return false;
        }
    }
    c->val = v;
    st_release_gpu(&c->seq, pos + 1);
    q_avail_add(q, 1);
    return true;
}

// Non-blocking pop: 1 with *out set, 0 when the queue is empty, -1 when the
// cell of a reserved position was not published within `limit_ns` (an error:
// the caller reports it).
__device__ __forceinline__ int q_try_pop(QueueHdr *q, QCell *cells, uint32_t *out, uint64_t limit_ns) {
    if (q_avail(q) <= 0) return 0;
    if (q_avail_add(q, -1) <= 0) {
        q_avail_add(q, 1);
        return 0;
    }
    const uint64_t pos = add_u64(&q->deq, 1);
    QCell *c = &cells[pos & q->mask];
    if (ld_acquire_gpu(&c->seq) != pos + 1) {
        WaitClock w(limit_ns);
        while (ld_acquire_gpu(&c->seq) != pos + 1) {
            if (!w.again()) return -1;
        }
    }
    *out = *((volatile uint32_t *)&c->val);
    st_release_gpu(&c->seq, pos + (uint64_t)q->mask + 1);
    return 1;
}

// Items published and not yet reserved (for scheduling decisions only).
__device__ __forceinline__ int64_t q_len(QueueHdr *q) { return q_avail(q); }

}  // namespace cafgpu
