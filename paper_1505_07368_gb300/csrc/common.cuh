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
// Bounded MPMC queue (array of cells with sequence numbers; a push reserves a
// position with one atomic add, a pop claims the head with one CAS).  Each
// value is in the queue at most once per push; capacity is a power of two and
// is sized by the host so that a push never needs to wait for space except
// for the short window in which a popper has claimed the cell but not yet
// released it.
// ---------------------------------------------------------------------------
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
    return true;
}

// Non-blocking pop: false when the queue is empty.
__device__ __forceinline__ bool q_try_pop(QueueHdr *q, QCell *cells, uint32_t *out) {
    uint64_t pos = ld_relaxed_gpu(&q->deq);
    for (int tries = 0; tries < 64; ++tries) {
        QCell *c = &cells[pos & q->mask];
        uint64_t seq = ld_acquire_gpu(&c->seq);
        int64_t diff = (int64_t)(seq - (pos + 1));
        if (diff == 0) {
            uint64_t prev = cas_u64(&q->deq, pos, pos + 1);
            if (prev == pos) {
                uint32_t v = *((volatile uint32_t *)&c->val);
                st_release_gpu(&c->seq, pos + (uint64_t)q->mask + 1);
                *out = v;
                return true;
            }
            pos = prev;
        } else if (diff < 0) {
            return false;
        } else {
            pos = ld_relaxed_gpu(&q->deq);
        }
    }
    return false;
}

// Approximate length (for scheduling decisions only).
__device__ __forceinline__ int64_t q_len(QueueHdr *q) {
    return (int64_t)(ld_relaxed_gpu(&q->enq) - ld_relaxed_gpu(&q->deq));
}

}  // namespace cafgpu
