// The persistent drain kernel and the other device entry points of the
// runtime (per-message launches, prime-table sieve, actor reset).
//
// Actor model mapping (Sec. 3.2 mailbox, Sec. 6 scheduler):
//
//  * Mailbox: each actor owns a power-of-two ring of 64-byte slots in HBM.
//    Enqueue takes a ticket with one atomic add on the actor's tail, writes
//    the slot and publishes it with a release store of seq = ticket + 1; a
//    warp enqueueing several messages for one actor takes one ticket block,
//    lanes in send order.  Only the current claim holder dequeues, so the
//    head needs no atomics (the single-reader property of Sec. 3.2).
//  * Scheduler: an actor that receives a message while WAITING becomes READY
//    and its id is pushed to a global ready queue (the paper's
//    central/internal enqueue).  A worker warp pops it, marks it RUNNING,
//    dequeues up to the per-claim limit (the max_msgs knob of Sec. 6.1),
//    and either re-queues it (resume_job_later) or parks it as WAITING.
//  * Payloads: stateful ring actors are run by the claiming warp, one message
//    at a time.  Factorization actors are pure: the claim moves up to K
//    messages into a batch record and pushes W work items; any warp may run
//    an item, and the last one to finish writes the replies in mailbox order.
//
// Every wait is bounded (WaitClock); when a limit expires the kernel records
// an error code, sets the exit flag and all warps return.
#include <cuda_runtime.h>

#include "common.cuh"
#include "factor.cuh"
#include "gemm_packed.cuh"
#include "layout.h"
#include "mandel.cuh"

namespace cafgpu {

constexpr uint32_t FULL = 0xFFFFFFFFu;

struct MsgData {
    uint64_t payload;
    uint64_t reply_addr;
    uint64_t tag;
    uint32_t sender, sender_seq, kind, reply_token;
};

__device__ __forceinline__ bool exit_requested(const DevCtl *ctl) {
    return *((volatile const uint32_t *)&ctl->exit_flag) != 0 ||
           *((volatile const uint32_t *)&ctl->error_word) != 0;
}

__device__ __forceinline__ void fail(const DrainParams &P, uint32_t code, uint32_t site, uint64_t d0 = 0,
                                     uint64_t d1 = 0) {
    if (atomicCAS(reinterpret_cast<unsigned int *>(&P.ctl->error_word), 0u, code | (site << 8)) == 0u) {
        P.ctl->diag[0] = d0;
        P.ctl->diag[1] = d1;
    }
    if (P.hctl) st_release_sys(&P.hctl->error_word, *((volatile uint32_t *)&P.ctl->error_word));
    atomicExch(reinterpret_cast<unsigned int *>(&P.ctl->exit_flag), 1u);
}

// A work item names an existing job record and one of its tiles, pack panels
// or bands.
__device__ bool work_item_ok(const DrainParams &P, uint32_t item);

// Validation mode: indices taken from queues, messages and records are checked
// against their arrays before they are used.  A failed check records
// kErrBounds (the site, the index and the limit) and the kernel unwinds as
// after an expired wait; nothing out of range is read or written.
__device__ __forceinline__ bool actor_ok(const DrainParams &P, uint32_t a) {
    return a < P.n_actors || (P.fork_pool && a - P.fork_base < P.fork_pool);
}
__device__ __noinline__ void bounds_fail(const DrainParams &P, uint32_t site, uint64_t idx, uint64_t lim) {
    fail(P, kErrBounds, site, idx, lim);
}
// Actor `a` and its whole mailbox lie inside the actor table and slot pool.
__device__ __forceinline__ bool mailbox_ok(const DrainParams &P, uint32_t a) {
    if (!actor_ok(P, a)) return false;
    const ActorDesc *A = &P.actors[a];
    return A->slot_base + (uint64_t)A->cap_mask < P.n_slots;
}

__device__ __forceinline__ void heartbeat(const DrainParams &P) {
    *((volatile uint64_t *)&P.ctl->heartbeat) = globaltimer();
}

// Ready actors (Sec. 6.2: the scheduler).  By default one global queue.  With
// work stealing (P.steal) every CTA has its own queue: the actors a CTA wakes
// go to its queue (to the global one when it is nearly full), and a worker
// pops its CTA's queue first, then the global one (host messages, overflow),
// then tries a few other CTAs' queues.  Only the owning CTA pushes to a local
// queue, so kLocalQueueSlack bounds the pushes in flight past the check.
__device__ __forceinline__ bool ready_push(const DrainParams &P, uint32_t a) {
    if (P.steal) {
        QueueHdr *q = &P.localq_hdr[blockIdx.x];
        const uint64_t used = ld_relaxed_gpu(&q->enq) - ld_relaxed_gpu(&q->deq);
        if (used + kLocalQueueSlack < P.localq_cap)
            return q_push(q, P.localq + (size_t)blockIdx.x * P.localq_cap, a, P.wait_limit_ns);
    }
    return q_push(&P.ctl->readyq, P.readyq, a, P.wait_limit_ns);
}

// Steal an actor from up to kStealTries random other CTAs' queues.
__device__ __noinline__ int ready_steal(const DrainParams &P, uint32_t *a, uint32_t &rng) {
    for (uint32_t k = 0; k < kStealTries; ++k) {
        rng = rng * 1664525u + 1013904223u;
        const uint32_t v = (rng >> 8) % gridDim.x;
        if (v == blockIdx.x) continue;
        const int ps = q_try_pop(&P.localq_hdr[v], P.localq + (size_t)v * P.localq_cap, a, P.wait_limit_ns);
        if (ps != 0) return ps;
    }
    return 0;
}

// Lane 0: the next ready actor (1), none (0), or an expired wait (-1).  `rng`
// is the caller's victim generator (a linear congruential step per try).
__device__ int ready_pop(const DrainParams &P, uint32_t *a, uint32_t &rng) {
    if (P.steal) {
        const int pr = q_try_pop(&P.localq_hdr[blockIdx.x], P.localq + (size_t)blockIdx.x * P.localq_cap, a,
                                 P.wait_limit_ns);
        if (pr != 0) return pr;
    }
    const int pr = q_try_pop(&P.ctl->readyq, P.readyq, a, P.wait_limit_ns);
    if (pr != 0 || !P.steal || gridDim.x < 2) return pr;
    return ready_steal(P, a, rng);
}

// Warp-collective enqueue: every lane with `valid` holds one message for
// actor `a`; lanes are in send order.  Messages that fit are published, the
// receiver is woken, and only then do lanes whose slot is still occupied wait
// for the receiver to make room (waking first keeps a full mailbox from
// waiting on a consumer that was never scheduled).  Returns false (all
// lanes) on a wait that expired.
// With `handoff` set, a receiver this call wakes is not queued: its id is
// returned through *handoff (kNone if none was woken) and the caller runs it
// next -- the paper's internal enqueue, which puts an actor readied by a
// worker at the front of that worker's own queue.  Only for single-lane sends.
__device__ bool warp_enqueue(const DrainParams &P, bool valid, uint32_t a, const MsgData &m,
                             uint32_t *handoff = nullptr) {
    const uint32_t lane = lane_id();
    const uint32_t vmask = __ballot_sync(FULL, valid);
    if (!vmask) return true;
    if (P.validation) {
        const bool bad = valid && !mailbox_ok(P, a);
        if (__any_sync(FULL, bad)) {
            if (bad) bounds_fail(P, 40, a, P.n_slots);
            return false;
        }
    }
    if (lane == 0) add_u64(&P.ctl->ingested, __popc(vmask));
    __syncwarp();
    const uint32_t key = valid ? a : 0xFFFFFFFFu;
    uint32_t peers = __match_any_sync(FULL, key) & vmask;
    const int leader = valid ? __ffs(peers) - 1 : (int)lane;
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    uint64_t t0 = 0;
    ActorDesc *A = valid ? &P.actors[a] : nullptr;
    if (valid && (int)lane == leader) t0 = add_u64(&A->tail, __popc(peers));
    t0 = __shfl_sync(FULL, t0, leader);
    const uint64_t t = t0 + rank;
    const uint32_t mask = valid ? A->cap_mask : 0;
    bool pending = valid;
    WaitClock w(P.wait_limit_ns);
    for (;;) {
        // acquire: pairs with the consumer's release of head, so the slot's
        // previous message has been read before this write replaces it
        bool published = false;
        if (pending && t - ld_acquire_gpu(&A->head) <= mask) {
            Slot *s = &P.slots[A->slot_base + (t & mask)];
            // the slot's fields in three stores (bytes 8, 16..31, 32..47)
            s->payload = m.payload;
            *reinterpret_cast<ulonglong2 *>(&s->reply_addr) = make_ulonglong2(m.reply_addr, m.tag);
            *reinterpret_cast<uint4 *>(&s->sender) = make_uint4(m.sender, m.sender_seq, m.kind, m.reply_token);
            st_release_gpu(&s->seq, t + 1);
            pending = false;
            published = true;
        }
        // wake a receiver to which this round published (fence: Dekker
        // pattern with release_actor).  A round that published nothing has
        // nothing to wake for: its lanes wait for room in a full mailbox,
        // whose receiver is ready or running.  The state is read first and
        // only a WAITING receiver is CASed: either this read sees WAITING, or
        // the receiver's release sees the tail these tickets advanced.
        __syncwarp();   // every lane's slot writes before the leader's state check
        const uint32_t pubm = __ballot_sync(FULL, published);
        bool qok = true;
        bool woke = false;
        if (pubm) {
            asm volatile("fence.sc.gpu;" ::: "memory");
            if (valid && (int)lane == leader && (pubm & peers) && ld_relaxed_gpu(&A->state) == kWaiting) {
                if (cas_acq_rel_gpu(&A->state, kWaiting, kReady) == kWaiting) {
                    if (handoff) woke = true;
                    else qok = ready_push(P, a);
                }
            }
        }
        if (handoff) {
            const uint32_t wm = __ballot_sync(FULL, woke);
            if (wm) *handoff = __shfl_sync(FULL, a, __ffs(wm) - 1);
        }
        if (!__all_sync(FULL, qok)) {
            if (!qok) fail(P, kErrWaitQueue, 2, P.ctl->readyq.enq, a);
            return false;
        }
        if (!__any_sync(FULL, pending)) return true;
        bool expired = false;
        if (pending) expired = !w.again();
        if (__any_sync(FULL, expired)) {
            if (expired) fail(P, kErrWaitSpace, 1, t, ((uint64_t)a << 32) | 1);
            return false;
        }
    }
}

// Park or re-queue an actor after its claim (warp-collective; lane 0 acts).
// The warp barrier orders every lane's slot reads before lane 0's release
// store of the new head: a producer that sees that head (acquire) may
// overwrite those slots.  The store of WAITING is a release as well, so a
// producer whose acquire-CAS wakes the actor passes the head on to the next
// claim through the ready queue.  `done`: 1 if the caller knows the actor has
// terminated, 0 if it knows it has not, -1 to read its state.  `moved`: false
// when the claim took no slot (the head keeps its value and needs no store).
__device__ void release_actor(const DrainParams &P, uint32_t a, uint64_t new_head, int done = -1,
                              bool moved = true, bool head_known = true) {
    __syncwarp();
    if (lane_id() == 0) {
        ActorDesc *A = &P.actors[a];
        if (moved) st_release_gpu(&A->head, new_head);
        if (done < 0) done = *((volatile uint32_t *)&A->state) == kDone;
        if (!done) {
            st_release_gpu(&A->state, kWaiting);
            asm volatile("fence.sc.gpu;" ::: "memory");
            // (a claim that did not read the head reads it here, beside the
            // tail: only the claim holder moves it)
            const uint64_t hd = head_known ? new_head : ld_relaxed_gpu(&A->head);
            if (ld_relaxed_gpu(&A->tail) != hd &&
                cas_u32(&A->state, kWaiting, kReady) == kWaiting) {
                if (!ready_push(P, a)) fail(P, kErrWaitQueue, 3);
            }
        }
    }
    __syncwarp();
}

// Validation mode: record the handling of `take` messages of actor `a` (lane i
// holds message i) in the log, in handling order (warp-collective).
__device__ void log_rows(const DrainParams &P, uint32_t a, uint32_t take, const MsgData &m) {
    const uint32_t lane = lane_id();
    uint64_t base = 0;
    if (lane == 0) base = add_u64(&P.ctl->log_count, take);
    base = __shfl_sync(FULL, base, 0);
    if (lane < take && base + lane < P.log_capacity) {
        LogRow *r = &P.log[base + lane];
        r->actor = a;
        r->sender = m.sender;
        r->sender_seq = m.sender_seq;
        r->kind = m.kind;
        r->stamp = base + lane;
        r->tag = m.tag;
        r->value = m.payload;
    }
}

// Dequeue from the claimed actor: of the next `want` (<= 32) tickets, take
// the run of consecutive published slots starting at `head` (lane i reads
// slot head + i).  A ticket may be taken before its slot is published, and a
// producer may be waiting for room behind it, so only published slots are
// taken; if none is, wait (bounded) for the first.  Returns the number taken,
// 0 after an expired wait.
__device__ uint32_t warp_dequeue(const DrainParams &P, uint32_t a, uint64_t head, uint32_t want,
                                 MsgData &m) {
    const uint32_t lane = lane_id();
    if (P.validation && !mailbox_ok(P, a)) {
        if (lane == 0) bounds_fail(P, 41, a, P.n_slots);
        return 0;
    }
    ActorDesc *A = &P.actors[a];
    const uint64_t t = head + lane;
    Slot *s = &P.slots[A->slot_base + (t & A->cap_mask)];
    bool pub = lane < want && ld_acquire_gpu(&s->seq) == t + 1;
    uint32_t pm = __ballot_sync(FULL, pub);
    if (!(pm & 1u)) {
        bool ok = true;
        if (lane == 0) {
            WaitClock w(P.wait_limit_ns);
            while (ld_acquire_gpu(&s->seq) != t + 1) {
                if (!w.again()) { ok = false; break; }
            }
            if (!ok) fail(P, kErrWaitSlot, 4, t + 1, ld_acquire_gpu(&s->seq));
        }
        if (!__shfl_sync(FULL, ok, 0)) return 0;
        pub = lane < want && ld_acquire_gpu(&s->seq) == t + 1;
        pm = __ballot_sync(FULL, pub) | 1u;
    }
    const uint32_t take = (pm == FULL) ? 32u : (uint32_t)(__ffs(~pm) - 1);
    if (lane < take) {
        m.payload = s->payload;
        const ulonglong2 rt = *reinterpret_cast<const ulonglong2 *>(&s->reply_addr);
        const uint4 sk = *reinterpret_cast<const uint4 *>(&s->sender);
        m.reply_addr = rt.x;
        m.tag = rt.y;
        m.sender = sk.x;
        m.sender_seq = sk.y;
        m.kind = sk.z;
        m.reply_token = sk.w;
    }
    if (P.validation) log_rows(P, a, take, m);
    return take;
}

// SINK `a`'s wide take (outside validation mode): of the next `want` (<= 128)
// tickets, take the run of consecutive published slots starting at `head`;
// lane i reads slots head + i + 32 j (j < 4), so one round of loads covers
// 128 slots.  Each taken message is handled as the SINK's (count + its
// position + 1)-th: its reply is written and its value added to the lane's
// *vsum.  Returns the number taken, 0 if the slot at head is not published
// yet (the caller then takes the waiting 32-wide path).
__device__ __noinline__ uint32_t sink_take_wide(const DrainParams &P, uint32_t a, uint64_t head, uint32_t want,
                                                uint64_t count, uint64_t *vsum) {
    const uint32_t lane = lane_id();
    const ActorDesc *A = &P.actors[a];
    const uint64_t base = A->slot_base, cmask = A->cap_mask;
    uint32_t take = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        const uint64_t t = head + lane + 32 * j;
        const bool pub = lane + 32 * j < want && ld_acquire_gpu(&P.slots[base + (t & cmask)].seq) == t + 1;
        const uint32_t pm = __ballot_sync(FULL, pub);
        if (take == 32 * j) take += (pm == FULL) ? 32u : (uint32_t)(__ffs(~pm) - 1);
    }
    // the four slots' values and reply addresses in one round of loads
    uint64_t x[4], ra[4];
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        const uint32_t i = lane + 32 * j;
        const Slot *sl = &P.slots[base + ((head + i) & cmask)];
        x[j] = i < take ? sl->payload : 0;
        ra[j] = i < take ? sl->reply_addr : 0;
    }
    uint64_t v = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        v += x[j];
        if (ra[j]) {
            const Slot *sl = &P.slots[base + ((head + lane + 32 * j) & cmask)];
            write_reply(ra[j], 0, count + lane + 32 * j + 1, x[j], sl->tag, sl->reply_token);
        }
    }
    *vsum = v;
    return take;
}

// ---------------------------------------------------------------------------
// Factorization batches
// ---------------------------------------------------------------------------
__device__ void finalize_batch(const DrainParams &P, uint32_t b) {
    const uint32_t lane = lane_id();
    FactorBatch *B = &P.batches[b];
    __threadfence();
    const uint32_t cnt = B->count;
    if (lane < cnt) {
        const uint64_t n = B->n[lane];
        const uint32_t found = *((volatile uint32_t *)&B->found[lane]);
        int32_t st;
        uint64_t r0, r1;
        factor_result(n, (B->even_mask >> lane) & 1u, found, B->pbound[lane], P.primes, &st, &r0, &r1);
        write_reply(B->reply_addr[lane], st, r0, r1, B->tag[lane], B->reply_token[lane]);
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        add_u64(&P.ctl->messages, cnt);
        add_u64(&P.ctl->completed, cnt);
        if (!q_push(&P.ctl->freeq, P.freeq, b, P.wait_limit_ns)) fail(P, kErrWaitQueue, 5);
    }
    __syncwarp();
}

// Remove from the warp every slot whose bit is set in `mask` (highest first).
__device__ __forceinline__ void sweep_remove_mask(SweepRegs &s, uint32_t mask) {
    while (mask) {
        const int j = 31 - __clz(mask);
        mask &= ~(1u << j);
        sweep_remove(s, j);
    }
}

// Per-slot value v of the held slot at position `lane` (lane j of `v` holds
// the value of batch message j); 0xFFFFFFFF for lanes past the held slots.
__device__ __forceinline__ uint32_t held_value(const SweepRegs &s, uint32_t v) {
    const uint32_t lane = lane_id();
    const uint32_t x = __shfl_sync(FULL, v, slot_id(s, lane & 15u));
    return (int)lane < s.k ? x : 0xFFFFFFFFu;
}

// Smallest bound among the held slots (pb: lane j holds message j's bound).
__device__ __forceinline__ uint32_t sweep_min_bound(const SweepRegs &s, uint32_t pb) {
    return __reduce_min_sync(FULL, held_value(s, pb));
}

// CTA barrier over the first `nthreads` threads' warps.  Callers reach it
// right after lane-0-only blocks, so the warp is reconverged first and the
// non-aligned barrier form is used (bar.sync is barrier.sync.aligned, which
// requires the whole warp to execute it together).
__device__ __forceinline__ void named_bar_sync(uint32_t id, uint32_t nthreads) {
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait on an mbarrier phase; false (and an error recorded) on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(const DrainParams &P, uint64_t *bar, uint32_t parity,
                                                  uint32_t site) {
    if (mbar_try_wait(bar, parity)) return true;
    WaitClock wc(P.wait_limit_ns);
    while (!mbar_try_wait(bar, parity)) {
        if (!wc.again()) {
            fail(P, kErrWaitTable, site, parity, 0);
            return false;
        }
    }
    return true;
}

// Table producer (one lane of the producer warp): streams tiles 0, 1, ... of
// the prime table into the CTA ring until the group's bound is reached or no
// consumer holds a message, then ends the stream with a tile that carries no
// data (its full barrier is completed by a plain arrive; final_tile marks it).
// `t` counts ring tiles over the whole kernel; stage = t % kStages, use = t / kStages.
__device__ void group_produce(const DrainParams &P, GroupShared &G, TableTile *ring, uint32_t &t) {
    const uint32_t limit = G.limit_tiles;
    bool ok = true;
    for (uint32_t i = 0;; ++i, ++t) {
        const uint32_t st = t % kStages;
        const uint32_t use = t / kStages;
        if (use >= 1 && ok) ok = mbar_wait_bounded(P, &G.empty[st], (use - 1) & 1u, 12);
        if (!ok || i >= limit || *((volatile uint32_t *)&G.active) == 0) {
            *((volatile uint32_t *)&G.final_tile) = i;
            mbar_arrive(&G.full[st]);
            ++t;
            return;
        }
        const uint32_t i0 = i * kTile;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&G.full[st], 3 * kTile * 4);
        bulk_g2s(ring[st].p, P.primes + i0, kTile * 4, &G.full[st]);
        bulk_g2s(ring[st].pinv, P.pinv + i0, kTile * 4, &G.full[st]);
        bulk_g2s(ring[st].plim, P.plim + i0, kTile * 4, &G.full[st]);
    }
}

// Table producer (one lane of the producer warp): streams, in increasing
// order, every table tile some team of the group needs, until none is needed
// or no consumer holds a message.  Tile i is needed by a team whose batch
// reaches it and, for a segment s of a batch split into S, has i % S == s.
// Without split batches this is tiles 0, 1, ... up to the largest bound.
// Each stage carries its tile index; the stream ends with a stage that
// carries kNone and no data (its full barrier is completed by a plain
// arrive).  `t` counts ring tiles over the whole kernel; stage = t % kStages,
// use = t / kStages.
__device__ void group_produce_split(const DrainParams &P, GroupShared &G, TableTile *ring, uint32_t &t,
                              uint32_t n_cons, uint32_t wpb) {
    uint32_t tS[kConsumerWarps], ts[kConsumerWarps], tl[kConsumerWarps];
    uint32_t nt = 0, lim = 0;
    bool split = false;
    for (uint32_t tb = 0; (tb + 1) * wpb <= n_cons; ++tb) {
        const uint32_t enc = G.batch[tb * wpb];
        if (enc == kNone) continue;
        const FactorBatch *B = &P.batches[enc & 0xFFFFFFu];
        const uint32_t S = B->segs > 1 ? B->segs : 1u;
        tS[nt] = S;
        ts[nt] = (enc >> 24) % S;
        tl[nt] = (B->maxbound + kTile - 1) / kTile;
        lim = max(lim, tl[nt]);
        split |= S > 1;
        ++nt;
    }
    bool ok = true;
    uint32_t cur = 0;
    for (;; ++t) {
        const uint32_t st = t % kStages;
        const uint32_t use = t / kStages;
        if (use >= 1 && ok) ok = mbar_wait_bounded(P, &G.empty[st], (use - 1) & 1u, 12);
        uint32_t idx = kNone;
        if (ok && *((volatile uint32_t *)&G.active) != 0) {
            if (!split) {
                if (cur < lim) idx = cur;
            } else {
                for (uint32_t k = 0; k < nt; ++k) {
                    const uint32_t i = cur + (ts[k] + tS[k] - cur % tS[k]) % tS[k];   // first i >= cur in segment
                    if (i < tl[k] && i < idx) idx = i;
                }
            }
        }
        *((volatile uint32_t *)&G.tile_idx[st]) = idx;
        if (idx == kNone) {
            mbar_arrive(&G.full[st]);
            ++t;
            return;
        }
        cur = idx + 1;
        const uint32_t i0 = idx * kTile;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&G.full[st], 3 * kTile * 4);
        bulk_g2s(ring[st].p, P.primes + i0, kTile * 4, &G.full[st]);
        bulk_g2s(ring[st].pinv, P.pinv + i0, kTile * 4, &G.full[st]);
        bulk_g2s(ring[st].plim, P.plim + i0, kTile * 4, &G.full[st]);
    }
}

// Consumer warp: sweep held batch `enc` ((segment << 24) | batch record;
// kNone: only keep the ring moving) over the streamed tiles of its segment.
// A team of `wpb` warps shares one batch; member `r` tests the chunks u of
// each tile with u % wpb == r, and members drop messages that another member,
// of any segment, has already decided below their position.  (A segment may
// see tiles past its messages' bounds that another team needs: they are
// tested only until the bound check drops the messages, and a hit at or past
// a message's bound is no divisor below its square root.)
constexpr uint32_t kTopUpTries = 8;    // further actors a factor claim may take messages from
constexpr uint32_t kSweepPrimes = 4;   // chunks (primes per lane) tested per step
static_assert((kTile / 32) % (kSweepPrimes * kConsumerWarps) == 0, "a tile splits into steps for any team size");

// kSplit: the drain splits batches (the stream carries tile indices); else
// the sequential stream of group_produce, whose end is G.final_tile.
template <bool kSplit>
__device__ void group_consume(const DrainParams &P, GroupShared &G, const TableTile *ring, uint32_t &t,
                              uint32_t enc, uint32_t r, uint32_t wpb) {
    const uint32_t lane = lane_id();
    const uint32_t b = (!kSplit || enc == kNone) ? enc : (enc & 0xFFFFFFu);
    FactorBatch *B = (b != kNone) ? &P.batches[b] : nullptr;
    uint32_t segs = 1, seg = 0;
    if constexpr (kSplit) {
        segs = (B && B->segs > 1) ? B->segs : 1u;
        seg = enc == kNone ? 0u : (enc >> 24) % segs;
    }
    SweepRegs s;
    sweep_init(s);
    if (B) {
        const uint32_t cnt = B->count;
#pragma unroll
        for (int j = 0; j < (int)kFactorKMax; ++j) {
            if (j < (int)cnt) {
                const bool even = (B->even_mask >> j) & 1u;
                if (B->pbound[j] > 0 && !even) {
                    const uint64_t n = B->n[j];
#pragma unroll
                    for (int i = 0; i <= j; ++i)
                        if (i == s.k) sweep_set(s, i, n);
                    s.ids |= (uint64_t)j << (4 * s.k);
                    ++s.k;
                }
            }
        }
    }
    bool counted = B != nullptr;   // included in G.active
    if (counted && s.k == 0) {
        if (lane == 0) atomicSub(&G.active, 1u);
        counted = false;
    }
    // bounds of the batch's messages, lane j holding message j's
    const uint32_t pbv = (B && lane < B->count) ? B->pbound[lane] : 0xFFFFFFFFu;
    uint32_t next_drop = s.k > 0 ? sweep_min_bound(s, pbv) : 0xFFFFFFFFu;
    uint64_t tests = 0;
    for (uint32_t i = 0;; ++i, ++t) {
        const uint32_t st = t % kStages;
        const bool ok = mbar_wait_bounded(P, &G.full[st], (t / kStages) & 1u, 13);
        if (!__all_sync(FULL, ok)) break;
        uint32_t tile = i;
        if constexpr (kSplit) {
            tile = *((volatile uint32_t *)&G.tile_idx[st]);
            if (tile == kNone) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&G.empty[st]);
                ++t;
                break;
            }
        } else {
            const uint32_t fin = *((volatile uint32_t *)&G.final_tile);
            if (i >= fin) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&G.empty[st]);
                ++t;
                break;
            }
        }
        if (s.k > 0 && (!kSplit || segs == 1 || tile % segs == seg)) {
            const uint32_t start = tile * kTile;
            // teammates' hits (lane j: message j), read now and applied after
            // this tile so the load's latency overlaps the tests; a stale
            // value only costs tests
            // (other segments of a split batch record theirs in the same slots)
            const bool shared_found = wpb > 1 || (kSplit && segs > 1);
            uint32_t fv = 0xFFFFFFFFu;
            if (shared_found && lane < kFactorKMax) fv = ld_relaxed_gpu(&B->found[lane]);
            const uint32_t tbase = smem_u32(&ring[st]);
            uint32_t tile_tests = 0;
            // kSweepPrimes chunks per step, u + q wpb (kTile / 32 is a multiple
            // of kSweepPrimes * wpb); one copy of the body: the test switch is
            // large, and an unrolled tile loop overflows the instruction cache.
            // The held messages are read-only inside the step loop: a step
            // with a hit, or one that reaches the next bound, leaves the loop
            // and is finished outside it, so the loop carries no register
            // moves for the held slots.
            const uint32_t ustep = kSweepPrimes * wpb;
            const uint32_t qstride = wpb * 32 * 4;      // bytes between a lane's primes of one step
            uint32_t u = r;
            while (u < kTile / 32 && s.k > 0) {
                uint32_t pp[kSweepPrimes], pi[kSweepPrimes], pl[kSweepPrimes];
                const uint32_t k_now = (uint32_t)s.k;
                uint32_t steps = 0;
                bool hit = false, stop = false;
#pragma unroll 1
                for (;;) {
                    uint32_t addr = tbase + (u * 32 + lane) * 4;
#pragma unroll
                    for (uint32_t q = 0; q < kSweepPrimes; ++q, addr += qstride) {
                        pp[q] = lds_u32_at<0>(addr);
                        pi[q] = lds_u32_at<kTile * 4>(addr);
                        pl[q] = lds_u32_at<2 * kTile * 4>(addr);
                    }
                    ++steps;
                    hit = __any_sync(FULL, sweep_chunks<kSweepPrimes>(s, pp, pi, pl));
                    // the next step starts at c1 + 32 wpb
                    const uint32_t c1 = start + u * 32 + (kSweepPrimes - 1) * 32 * wpb;
                    if (hit || c1 + 32 * wpb >= next_drop) {
                        stop = true;
                        break;
                    }
                    u += ustep;
                    if (u >= kTile / 32) break;
                }
                tile_tests += steps * k_now * 32u * kSweepPrimes;
                if (!stop) break;
                // finish step u: its hits, then its bound check
                const uint32_t c0 = start + u * 32;
                if (hit) {
                    uint32_t h[kSweepPrimes], hh = 0;
#pragma unroll
                    for (uint32_t q = 0; q < kSweepPrimes; ++q) {
                        h[q] = sweep_which(s, pp[q], pi[q], pl[q]);
                        hh |= h[q];
                    }
                    const uint32_t any = __reduce_or_sync(FULL, hh);
                    for (uint32_t m = any; m; m &= m - 1) {
                        const int j = __ffs(m) - 1;
                        uint32_t x = 0xFFFFFFFFu;
#pragma unroll
                        for (uint32_t q = 0; q < kSweepPrimes; ++q)
                            if ((h[q] >> j) & 1u) x = min(x, c0 + q * 32 * wpb + lane);
                        const uint32_t mn = __reduce_min_sync(FULL, x);
                        if (lane == 0) atomicMin(reinterpret_cast<unsigned int *>(&B->found[slot_id(s, j)]), mn);
                    }
                    sweep_remove_mask(s, any);
                }
                const uint32_t c1 = c0 + (kSweepPrimes - 1) * 32 * wpb;
                if (s.k > 0 && c1 + 32 * wpb >= next_drop) {
                    const uint32_t rm = __ballot_sync(FULL, held_value(s, pbv) <= c1 + 32 * wpb);
                    sweep_remove_mask(s, rm);
                    next_drop = s.k > 0 ? sweep_min_bound(s, pbv) : 0xFFFFFFFFu;
                }
                u += ustep;
            }
            tests += tile_tests;
            // drop messages a teammate has factored below the next tile: this
            // warp's remaining primes cannot give a smaller divisor
            if (shared_found && s.k > 0) {
                const uint32_t rm = __ballot_sync(FULL, held_value(s, fv) < start + kTile);
                if (rm) {
                    sweep_remove_mask(s, rm);
                    next_drop = s.k > 0 ? sweep_min_bound(s, pbv) : 0xFFFFFFFFu;
                }
            }
            if (s.k == 0 && counted) {
                if (lane == 0) atomicSub(&G.active, 1u);
                counted = false;
            }
            if (lane == 0 && (i & 255u) == 0) heartbeat(P);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&G.empty[st]);
    }
    if (counted && lane == 0) atomicSub(&G.active, 1u);   // left early after an error
    if (B) {
        if (lane == 0) {
            add_u64(&P.ctl->prime_tests, tests);
            add_u64(&P.ctl->factor_items, 1);
        }
        uint32_t left = 0;
        if (lane == 0) {
            __threadfence();
            left = atomicSub(reinterpret_cast<unsigned int *>(&B->items_left), 1u);
        }
        left = __shfl_sync(FULL, left, 0);
        if (left == 1) finalize_batch(P, b);
    }
}

// Claim factor actor `a`: move up to cap - pos of its messages into a group
// of batch records, message q of the group at slot q % K of record q / K
// (lane r of `recs` holds the group's record r).  A batch may hold the
// messages of several actors: replies go to each message's own reply record,
// and each actor's messages enter in its mailbox order.  Releases the actor;
// returns the group's new message count.
__device__ uint32_t claim_factor_take(const DrainParams &P, uint32_t a, uint32_t recs, uint32_t pos,
                                      uint32_t cap) {
    const uint32_t lane = lane_id();
    const uint32_t K = P.factor_k;
    ActorDesc *A = &P.actors[a];
    if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
    __syncwarp();
    const uint64_t head = *((volatile uint64_t *)&A->head);
    const uint64_t tail = ld_acquire_gpu(&A->tail);
    uint32_t limit = cap - pos;
    if (P.max_claim && P.max_claim < limit) limit = P.max_claim;
    // at most one mailbox's worth: a sender holding a ticket past head + capacity
    // publishes only after this claim has released the head
    if (A->cap_mask < limit - 1) limit = A->cap_mask + 1;
    const uint64_t avail = tail - head;
    const uint32_t want = avail < limit ? (uint32_t)avail : limit;
    uint32_t took = 0;
    while (took < want) {
        const uint32_t w = min(want - took, 32u);
        MsgData m{};
        const uint32_t take = warp_dequeue(P, a, head + took, w, m);
        const uint32_t q = pos + took + lane;
        const uint32_t rec = __shfl_sync(FULL, recs, min(q / K, 31u));
        if (lane < take) {
            FactorBatch *B = &P.batches[rec];
            const uint32_t i = q % K;
            const uint64_t n = m.payload;
            const bool even = (n >= 4) && !(n & 1u);
            B->n[i] = n;
            B->pbound[i] = even ? 0 : factor_bound(P.primes, P.nprimes, n);
            B->found[i] = kNoFactor;
            B->reply_addr[i] = m.reply_addr;
            B->reply_token[i] = m.reply_token;
            B->tag[i] = m.tag;
        }
        took += take;
        if (take < w) break;
    }
    release_actor(P, a, head + took, 0);
    if (lane == 0) add_u64(&P.ctl->claims, 1);
    __syncwarp();
    return pos + took;
}

// Reorder the `count` messages of a claim's group of records by n, so that
// each batch holds messages of similar size.  A batch is swept until its
// last message is decided, and the smallest factor of a number tends to grow
// with the number, so batches of similar n leave fewer slots idle.  Lane e %
// 32 ranks messages e (ties by position), all fields are read, and after the
// warp barrier each is written to the slot of its rank (found is still
// kNoFactor everywhere).
constexpr uint32_t kGroupRecords = 16;    // batch records one factor claim may fill
constexpr uint32_t kGroupMessages = 256;  // messages one factor claim may take
__device__ __noinline__ void factor_group_sort(const DrainParams &P, uint32_t recs, uint32_t count) {
    const uint32_t lane = lane_id();
    const uint32_t K = P.factor_k;
    constexpr int J = kGroupMessages / 32;
    uint64_t key[J];
    uint32_t rank[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t e = lane + 32u * j;
        const uint32_t rec = __shfl_sync(FULL, recs, min(e / K, 31u));
        key[j] = e < count ? P.batches[rec].n[e % K] : ~0ull;
        rank[j] = 0;
    }
#pragma unroll
    for (int jj = 0; jj < J; ++jj) {
        if (32u * jj >= count) break;
        for (uint32_t src = 0; src < 32; ++src) {
            const uint64_t kf = __shfl_sync(FULL, key[jj], src);
            const uint32_t f = src + 32u * jj;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const uint32_t e = lane + 32u * j;
                rank[j] += (f < count && (kf < key[j] || (kf == key[j] && f < e))) ? 1u : 0u;
            }
        }
    }
    // move the fields one at a time: each pass reads all its values before
    // the warp barrier and writes them after it
    uint32_t dst[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t e = lane + 32u * j;
        const uint32_t r = e < count ? rank[j] : 0u;
        dst[j] = __shfl_sync(FULL, recs, min(r / K, 31u)) * kFactorKMax + r % K;
    }
    auto slot_of = [&](uint32_t e) {
        return __shfl_sync(FULL, recs, min(e / K, 31u)) * kFactorKMax + e % K;
    };
#pragma unroll 1
    for (int f = 0; f < 5; ++f) {
        uint64_t v[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const uint32_t e = lane + 32u * j;
            const uint32_t src = slot_of(e);
            const FactorBatch *B = &P.batches[src / kFactorKMax];
            const uint32_t i = src % kFactorKMax;
            v[j] = key[j];
            if (e < count) {
                if (f == 1) v[j] = B->pbound[i];
                else if (f == 2) v[j] = B->reply_addr[i];
                else if (f == 3) v[j] = B->reply_token[i];
                else if (f == 4) v[j] = B->tag[i];
            }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const uint32_t e = lane + 32u * j;
            if (e < count) {
                FactorBatch *B = &P.batches[dst[j] / kFactorKMax];
                const uint32_t i = dst[j] % kFactorKMax;
                if (f == 0) B->n[i] = v[j];
                else if (f == 1) B->pbound[i] = (uint32_t)v[j];
                else if (f == 2) B->reply_addr[i] = v[j];
                else if (f == 3) B->reply_token[i] = (uint32_t)v[j];
                else B->tag[i] = v[j];
            }
        }
        __syncwarp();
    }
}

// Start the sweep of batch b holding `count` messages: record it, split it
// if it is large (kSplit), or answer it at once when no message needs a sweep.
// Returns b when the caller's team sweeps it, kNone otherwise.
template <bool kSplit>
__device__ uint32_t factor_batch_launch(const DrainParams &P, uint32_t b, uint32_t count) {
    const uint32_t lane = lane_id();
    FactorBatch *B = &P.batches[b];
    if (count == 0) {
        if (lane == 0) q_push(&P.ctl->freeq, P.freeq, b, P.wait_limit_ns);
        return kNone;
    }
    __threadfence_block();
    uint32_t pb = 0;
    bool even = false;
    if (lane < count) {
        const uint64_t n = B->n[lane];
        even = (n >= 4) && !(n & 1u);
        pb = B->pbound[lane];
    }
    const uint32_t even_mask = __ballot_sync(FULL, lane < count && even);
    const uint32_t maxb = __reduce_max_sync(FULL, lane < count ? pb : 0u);
    // split a large batch over the teams that would otherwise idle: the
    // device's teams against the batch records in use
    uint32_t segs = 1;
    const uint32_t tiles = (maxb + kTile - 1) / kTile;
    if (kSplit && P.split > 1 && tiles >= kSplitMinTiles) {
        int64_t in_use = 0;
        if (lane == 0) in_use = (int64_t)P.n_batches - q_len(&P.ctl->freeq);
        in_use = __shfl_sync(FULL, in_use, 0);
        const uint32_t teams = gridDim.x * (kConsumerWarps / P.factor_w);
        const uint32_t idle = in_use >= 1 ? teams / (uint32_t)in_use : teams;
        segs = min(min(min(P.split, kSplitMax), tiles / kSplitTilesPerSeg), idle);
        if (segs < 2) segs = 1;
    }
    if (lane == 0) {
        B->count = count;
        B->even_mask = even_mask;
        B->maxbound = maxb;
        B->segs = segs;
        B->items_left = P.factor_w * segs;
    }
    __syncwarp();
    if (maxb == 0) {
        finalize_batch(P, b);
        return kNone;
    }
    if (kSplit && segs > 1) {
        // the record is complete before any segment can be taken
        __threadfence();
        bool ok = true;
        if (lane >= 1 && lane < segs) ok = q_push(&P.ctl->segq, P.segq, (lane << 24) | b, P.wait_limit_ns);
        if (!__all_sync(FULL, ok)) {
            if (!ok) fail(P, kErrWaitQueue, 33);
            return kNone;
        }
    }
    return b;   // segment 0 for the claiming team
}

// ---------------------------------------------------------------------------
// Ring token actors (stateful; the claiming warp runs them one message at a
// time).  Reading of Sec. 5 "Mixed Operations Under Work Load": the token
// loses one per hop; an actor receiving 0 terminates and forwards 0 once
// unless its successor has terminated; the master sends one factorization
// request to its worker at the start and on each token v > 0 it receives.
// ---------------------------------------------------------------------------
__device__ bool ring_emit_factor(const DrainParams &P, uint32_t a) {
    ActorDesc *A = &P.actors[a];
    MsgData m{};
    bool valid = false;
    uint32_t worker = 0;
    if (lane_id() == 0 && (A->flags & kActorMaster)) {
        const uint32_t k = A->round;
        if (k < A->factor_count) {
            A->round = k + 1;
            valid = true;
            worker = A->worker;
            m.payload = reinterpret_cast<const uint64_t *>(A->factor_n)[k];
            m.reply_addr = A->factor_replies + (uint64_t)k * sizeof(Reply);
            m.reply_token = 1;
            m.tag = k;
            m.sender = 0x80000000u | a;
            m.sender_seq = k;
            m.kind = kFactor;
        }
    }
    worker = __shfl_sync(FULL, worker, 0);
    return warp_enqueue(P, valid, worker, m);
}

// A message handed from one ring actor's run straight to the next actor's,
// without going through a mailbox (all lanes hold the same copy).
// A carried token has no reply record, and its sequence number is its value,
// so only its payload, tag, sender and kind travel.
struct Carry {
    bool has;
    uint64_t payload, tag;
    uint32_t sender, kind;
    // the receiver's successor, and whether it is a plain ring member (no
    // flags), read beside the claim's CAS (neither changes while its ring runs)
    uint32_t next;
    bool plain;
    __device__ MsgData msg() const {
        MsgData m{};
        m.payload = payload;
        m.tag = tag;
        m.sender = sender;
        m.sender_seq = (uint32_t)payload;
        m.kind = kind;
        return m;
    }
};

// Counters of a chain of ring runs, kept in registers (warp-uniform) and
// added to the device counters every kTallyHops runs and at the chain's end.
// Besides statistics, they hold the chain's completions and the ingestion of
// the tokens it carried directly (sends through a mailbox count `ingested`
// at once).  A carried token is completed only by the same chain, so the two
// lag by the same amount, and a flush adds `ingested` before `completed`:
// the counters never show the drain quiescent while a token is in flight.
struct RingTally {
    uint32_t done, claims, sends, carried;
    uint32_t pend;     // lane i < npend: a carried actor whose release waits for the batch
    uint32_t npend;
};
constexpr uint32_t kTallyHops = 32;
// Carried runs leave their actor claimed (RUNNING) until kReleaseBatch of
// them are pending; one warp operation then releases them all: the state
// stores, one fence.sc, and each actor's head and tail check (re-queueing an
// actor that messages reached in the meantime: a sender that saw it RUNNING
// did not wake it).  The protocol is release_actor's, only later.
constexpr uint32_t kReleaseBatch = 8;
__device__ void ring_release_pending(const DrainParams &P, RingTally &tl) {
    if (tl.npend == 0) return;
    const uint32_t lane = lane_id();
    __syncwarp();
    ActorDesc *A = lane < tl.npend ? &P.actors[tl.pend] : nullptr;
    if (A) st_release_gpu(&A->state, kWaiting);
    asm volatile("fence.sc.gpu;" ::: "memory");
    if (A && ld_relaxed_gpu(&A->tail) != ld_relaxed_gpu(&A->head) &&
        cas_u32(&A->state, kWaiting, kReady) == kWaiting) {
        if (!ready_push(P, tl.pend)) fail(P, kErrWaitQueue, 3);
    }
    tl.npend = 0;
    tl.pend = kNone;
    __syncwarp();
}
__device__ void ring_tally_flush(const DrainParams &P, RingTally &tl) {
    if (lane_id() == 0 && (tl.done | tl.claims | tl.sends | tl.carried)) {
        // everything the counted messages did (their sends counted in
        // ingested) is ordered before they count as completed
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (tl.carried) {
            add_u64(&P.ctl->ingested, tl.carried);
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
        }
        if (tl.sends) add_u64(&P.ctl->device_sends, tl.sends);
        if (tl.claims) add_u64(&P.ctl->claims, tl.claims);
        if (tl.done) {
            add_u64(&P.ctl->messages, tl.done);
            add_u64(&P.ctl->completed, tl.done);
        }
    }
    tl.done = tl.claims = tl.sends = tl.carried = 0;
    __syncwarp();
}

// Send token v from ring actor `a` to its successor.  Direct handoff: if the
// successor is waiting, this warp claims it (CAS WAITING -> RUNNING) and
// carries the token to its run instead of writing a mailbox slot -- no
// ticket, no slot round trip, no wake handshake.  Messages already in the
// successor's mailbox come from other senders (a ring holds one token, so
// this actor has none there): the successor's release finds them and
// re-queues it, and messages of different senders have no order to keep.
// Otherwise the token goes through the mailbox (warp_enqueue), and a
// successor this call wakes is returned in *handoff to run next.
// In a ring that a RECREATE master creates, a token of value 0 carries its
// origin (the actor id + 1 in the payload's high word), and its tag names the
// ring, the incarnation and the receiver's position: master + 1 in bits 0..31,
// the incarnation in bits 32..39, the position in bits 40..63.
__device__ bool ring_forward(const DrainParams &P, uint32_t a, int32_t v, uint32_t *handoff, Carry *carry,
                             RingTally &tl, uint32_t origin1 = 0, uint32_t known_next = kNone,
                             uint32_t known_flags = kNone) {
    // (known_next / known_flags: the sender's successor and flags when the
    // caller has them, so their descriptor line is not read again)
    ActorDesc *A = &P.actors[a];
    const uint32_t next = known_next != kNone ? known_next : A->next;
    const uint32_t aflags = known_flags != kNone ? known_flags : A->flags;
    MsgData m{};
    m.payload = (uint64_t)(uint32_t)v | ((uint64_t)origin1 << 32);
    m.kind = kToken;
    m.sender = 0x80000000u | a;
    m.sender_seq = (uint32_t)v;
    if (aflags & (kActorRecreate | kActorLink)) {
        const bool master = (aflags & kActorRecreate) != 0;
        const uint32_t pos = master ? 0u : A->ring_pos;
        const uint32_t recv = pos + 1 == A->ring_len ? 0u : pos + 1;
        m.tag = (uint64_t)((master ? a : A->ring_master) + 1) | ((uint64_t)(A->ring_inc & 0xFFu) << 32) |
                ((uint64_t)recv << 40);
    }
    const uint32_t lane = lane_id();
    tl.sends += 1;
    if (carry && !carry->has && next != a) {
        // a successor this chain still holds is released first
        if (__any_sync(FULL, lane < tl.npend && tl.pend == next)) ring_release_pending(P, tl);
        bool direct = false;
        uint32_t f = 0;
        ActorDesc *N = &P.actors[next];
        if (lane == 0) {
            // claimed: the token is carried into the successor's run.  Messages
            // already in its mailbox (from other senders: a ring holds one
            // token, so this sender has none there) are found by the run's
            // release, which reads the head beside the tail and re-queues the
            // actor; messages of different senders have no order to keep.
            direct = cas_acq_rel_gpu(&N->state, kWaiting, kRunning) == kWaiting;
        } else if (lane == 1) {
            f = N->next;    // read while lane 0's CAS is in flight
        } else if (lane == 2) {
            f = (N->flags == 0 && N->kind == kToken) ? 1u : 0u;
        }
        if (__shfl_sync(FULL, direct, 0)) {
            tl.carried += 1;   // ingested at the chain's next tally flush
            carry->has = true;
            carry->payload = m.payload;
            carry->tag = m.tag;
            carry->sender = m.sender;
            carry->kind = m.kind;
            carry->next = __shfl_sync(FULL, f, 1);
            carry->plain = __shfl_sync(FULL, f, 2) != 0;
            *handoff = next;
            return true;
        }
    }
    return warp_enqueue(P, lane == 0, next, m, handoff);
}

// RECREATE master `a` (claimed by this warp): spawn the ring_len - 1 members
// of its next incarnation from the device actor pool (warp-collective).
// Member i (position i + 1) gets the next member as successor, the last one
// the master; the master's successor becomes member 0.  The records are
// complete before the caller's first send reaches any of them.
__device__ uint32_t fork_take_id(const DrainParams &P);

__device__ bool ring_spawn(const DrainParams &P, uint32_t a) {
    const uint32_t lane = lane_id();
    ActorDesc *A = &P.actors[a];
    const uint32_t L = A->ring_len, nl = L - 1, inc = A->ring_inc;
    const int32_t init = A->init_state;
    uint32_t prev_last = kNone, first = kNone;
    for (uint32_t c0 = 0; c0 < nl; c0 += 32) {
        const uint32_t i = c0 + lane;
        uint32_t id = kNone;
        if (i < nl) id = fork_take_id(P);
        if (__any_sync(FULL, i < nl && id == kNone)) return false;   // the expired wait is recorded
        const uint32_t succ = __shfl_down_sync(FULL, id, 1);
        if (i < nl) {
            ActorDesc *M = &P.actors[id];
            M->kind = kToken;
            M->flags = kActorLink;
            M->next = i + 1 == nl ? a : (lane < 31 ? succ : kNone);   // kNone: patched by the next chunk
            M->worker = kNone;
            M->factor_count = 0;
            M->round = 0;
            M->user_state = init;
            M->init_state = init;
            M->ring_master = a;
            M->ring_len = L;
            M->ring_pos = i + 1;
            M->ring_inc = inc;
            M->ring_live = 0;
            *((volatile uint32_t *)&M->state) = kWaiting;
        }
        if (c0 > 0 && lane == 0) P.actors[prev_last].next = id;
        const uint32_t last_lane = nl - 1 - c0 < 31 ? nl - 1 - c0 : 31u;
        prev_last = __shfl_sync(FULL, id, last_lane);
        if (c0 == 0) first = __shfl_sync(FULL, id, 0);
    }
    if (lane == 0) {
        A->next = first;
        A->ring_live = nl;
        add_u64(&P.ctl->device_spawns, nl);
    }
    __threadfence();
    __syncwarp();
    return true;
}

// RECREATE master `a`, its running incarnation over (every member has
// terminated): true if another incarnation is to run (its index is advanced),
// false if the master terminates now (warp-collective; lane 0 writes).
__device__ bool ring_incarnation_over(const DrainParams &P, uint32_t a) {
    ActorDesc *A = &P.actors[a];
    const bool more = A->ring_inc + 1 < A->fork_token;
    if (lane_id() == 0) {
        if (more) {
            A->ring_inc += 1;
        } else {
            A->ring_live = 0;
            *((volatile uint32_t *)&A->state) = kDone;
        }
    }
    __syncwarp();
    return more;
}

// Run the claimed ring actor `a`: first the message carried to it (`carry`,
// from its predecessor's run on this warp), then its mailbox.  Returns the
// successor this warp woke or claimed (to be run next by the same warp) or
// kNone; a token carried to that successor is left in `carry`.  With
// `direct` false every forward goes through the mailbox.
__device__ uint32_t run_ring_actor(const DrainParams &P, uint32_t a, Carry &carry, bool direct, RingTally &tl) {
    const uint32_t lane = lane_id();
    uint32_t handoff = kNone;
    ActorDesc *A = &P.actors[a];
    const bool carried = carry.has;
    uint64_t head, take;
    if (carried) {
        // claimed by the predecessor's forward: the mailbox's messages are
        // left to this claim's release, which re-queues the actor
        head = 0;
        take = 0;
    } else {
        if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
        __syncwarp();
        head = *((volatile uint64_t *)&A->head);
        const uint64_t tail = ld_acquire_gpu(&A->tail);
        take = tail - head;
        // tail counts tickets a sender may not have published yet; a ticket at or
        // past head + capacity waits for room that this claim only releases at
        // its end, so a claim never goes past one mailbox's worth
        if (take > (uint64_t)A->cap_mask + 1) take = (uint64_t)A->cap_mask + 1;
        if (P.max_claim && take > P.max_claim) take = P.max_claim;
    }
    tl.claims += 1;
    Carry out{};
    out.has = false;
    // a ring that a RECREATE master creates: the 0 stops by its origin, and a
    // member that terminates returns its record to the pool after this run
    const bool recreated = (A->flags & (kActorRecreate | kActorLink)) != 0;
    const bool is_master = (A->flags & kActorRecreate) != 0;
    bool link_ended = false;
    bool ended = false;        // the actor is DONE (found so, or terminated here)
    uint64_t handled = 0;      // messages handled, counted as completed after the release
    for (uint64_t i = 0; i < take + (carried ? 1 : 0); ++i) {
        MsgData m{};
        if (carried && i == 0) {
            m = carry.msg();
            if (P.validation) log_rows(P, a, 1, m);
        } else {
            if (warp_dequeue(P, a, head, 1, m) == 0) return kNone;
            m.payload = __shfl_sync(FULL, m.payload, 0);
            m.kind = __shfl_sync(FULL, m.kind, 0);
            m.reply_addr = __shfl_sync(FULL, m.reply_addr, 0);
            m.reply_token = __shfl_sync(FULL, m.reply_token, 0);
            m.tag = __shfl_sync(FULL, m.tag, 0);
            head += 1;
        }
        const int32_t v = (int32_t)(uint32_t)m.payload;
        // a carried message's receiver was WAITING when it was claimed
        const bool dead = (carried && i == 0) ? false
                                              : __shfl_sync(FULL, *((volatile uint32_t *)&A->state) == kDone, 0);
        ended |= dead;
        bool ok = true;
        bool rejected = false;
        Carry *cp = direct ? &out : nullptr;
        if (dead) {
            if (lane == 0) write_reply(m.reply_addr, 2, 0, 0, m.tag, m.reply_token);
        } else if (is_master && ((m.kind >> 16) & (kMsgStart | kMsgRingDone))) {
            // a RECREATE master starts its first incarnation on START (unless
            // a ring is running) and the next one when the running one's
            // members have all terminated, until incarnations in all have run
            const bool start = ((m.kind >> 16) & kMsgStart) != 0;
            bool run_next = false;
            if (start) {
                rejected = A->ring_live != 0;
                if (!rejected && lane == 0) {
                    A->sink_count = (uint64_t)(uint32_t)v;
                    A->ring_inc = 0;
                }
                run_next = !rejected;
            } else {
                run_next = ring_incarnation_over(P, a);
                ended = !run_next;
            }
            __syncwarp();
            if (run_next) {
                const int32_t v0 = (int32_t)(uint32_t)A->sink_count;
                ok = ring_spawn(P, a) && ring_emit_factor(P, a) && ring_forward(P, a, v0, &handoff, cp, tl);
            }
        } else if ((m.kind >> 16) & kMsgStart) {
            ok = ring_emit_factor(P, a) && ring_forward(P, a, v, &handoff, cp, tl);
        } else if (v > 0) {
            ok = ring_emit_factor(P, a) && ring_forward(P, a, v - 1, &handoff, cp, tl);
        } else if (recreated) {
            // the 0 went once around from its origin: stop before reaching it
            // again (the same actors as "unless the successor has terminated",
            // without reading a successor's record, which may already serve a
            // new actor)
            const uint32_t origin1 = (uint32_t)(m.payload >> 32) ? (uint32_t)(m.payload >> 32) : a + 1;
            if (!is_master && lane == 0) *((volatile uint32_t *)&A->state) = kDone;
            link_ended = !is_master;
            ended |= !is_master;
            if (A->next + 1 != origin1) {
                ok = ring_forward(P, a, 0, &handoff, cp, tl, origin1);
            } else if (!is_master) {
                // the 0 stops here: every other actor of the incarnation has
                // terminated, so tell the master (a send of this message, so
                // counted before the message completes)
                MsgData d{};
                d.kind = kToken | (kMsgRingDone << 16);
                d.sender = 0x80000000u | a;
                tl.sends += 1;
                ok = warp_enqueue(P, lane == 0, A->ring_master, d);
            } else if (ring_incarnation_over(P, a)) {
                // the master is the last to terminate: start the next incarnation
                const int32_t v0 = (int32_t)(uint32_t)A->sink_count;
                ok = ring_spawn(P, a) && ring_emit_factor(P, a) && ring_forward(P, a, v0, &handoff, cp, tl);
            } else {
                ended = true;
            }
        } else {
            if (lane == 0) *((volatile uint32_t *)&A->state) = kDone;
            ended = true;
            uint32_t succ_state = 0;
            if (lane == 0) succ_state = *((volatile uint32_t *)&P.actors[A->next].state);
            succ_state = __shfl_sync(FULL, succ_state, 0);
            if (succ_state != kDone) ok = ring_forward(P, a, 0, &handoff, cp, tl);
        }
        if (!ok) return kNone;
        if (rejected) {
            if (lane == 0) write_reply(m.reply_addr, 3, 0, 0, m.tag, m.reply_token);
        } else if (!dead && lane == 0 && !((m.kind >> 16) & kMsgRingDone)) {
            A->user_state = v;
            write_reply(m.reply_addr, 0, (uint64_t)(uint32_t)v, 0, m.tag, m.reply_token);
        }
        __syncwarp();
        ++handled;
    }
    if (carried && !ended) {
        // released with the chain's next batch
        if (lane == tl.npend) tl.pend = a;
        if (++tl.npend == kReleaseBatch) ring_release_pending(P, tl);
    } else {
        release_actor(P, a, head, ended ? 1 : 0, !carried, !carried);
    }
    // counted as completed at the chain's next tally flush (after its fence)
    tl.done += (uint32_t)handled;
    carry = out;
    if (link_ended && lane == 0) {
        // the claim is released and nothing more is sent to a terminated
        // member: its record goes back to the pool
        __threadfence();
        if (!q_push(&P.ctl->forkq, P.forkq, a, P.wait_limit_ns)) fail(P, kErrWaitQueue, 35);
    }
    __syncwarp();
    return handoff;
}

// Claim a ring actor and keep running the actors its messages wake, up to a
// bound, after which the next one goes back to the ready queue.
// A carried token cannot go back to the ready queue, so the last run of a
// chain forwards through the mailbox.
// The hop of a plain ring member (no flags) receiving a carried plain token
// v > 0 that needs no reply: the steps of its run in run_ring_actor (log,
// forward v - 1, record v, count, release with the chain's next batch)
// without the general run's dispatch.  Returns false, having done nothing,
// for any other run.
__device__ bool ring_fast_hop(const DrainParams &P, uint32_t &cur, Carry &carry, bool direct, RingTally &tl) {
    const uint32_t lane = lane_id();
    const uint32_t a = cur;
    ActorDesc *A = &P.actors[a];
    const int32_t v = (int32_t)(uint32_t)carry.payload;
    if (!direct || !carry.plain || carry.kind != kToken || v <= 0) return false;
    tl.claims += 1;
    if (P.validation) log_rows(P, a, 1, carry.msg());
    Carry out{};
    out.has = false;
    uint32_t handoff = kNone;
    if (!ring_forward(P, a, v - 1, &handoff, &out, tl, 0, carry.next, 0u)) {
        cur = kNone;
        return true;
    }
    if (lane == 0) A->user_state = v;
    __syncwarp();
    tl.done += 1;
    if (lane == tl.npend) tl.pend = a;
    if (++tl.npend == kReleaseBatch) ring_release_pending(P, tl);
    carry = out;
    cur = handoff;
    return true;
}

__device__ void claim_ring(const DrainParams &P, uint32_t a) {
    constexpr int kMaxChain = 1 << 14;
    uint32_t cur = a;
    Carry carry{};
    carry.has = false;
    RingTally tl{0, 0, 0, 0, kNone, 0};
    for (int i = 0; cur != kNone && i < kMaxChain && ((i & 7) != 0 || !exit_requested(P.ctl)); ++i) {
        const bool direct = i + 1 < kMaxChain;
        if (!(carry.has && ring_fast_hop(P, cur, carry, direct, tl))) cur = run_ring_actor(P, cur, carry, direct, tl);
        if ((i & 255) == 0 && lane_id() == 0) heartbeat(P);
        if ((uint32_t)(i + 1) % kTallyHops == 0) ring_tally_flush(P, tl);
    }
    ring_release_pending(P, tl);
    ring_tally_flush(P, tl);
    if (cur != kNone && lane_id() == 0 && !ready_push(P, cur))
        fail(P, kErrWaitQueue, 18);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// SINK and SOURCE actors: the two ends of the paper's N:1 mailbox experiment
// (Sec. 5, "Mailbox Performance in N:1 Communication Scenario").
// ---------------------------------------------------------------------------
constexpr uint32_t kSinkChunk = 4096;     // messages a SINK handles per claim
constexpr uint32_t kSourceChunk = 1024;   // messages a SOURCE sends per run

// Warp sum of a 64-bit value (all lanes).
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Claimed SINK `a`: take up to kSinkChunk messages, 32 per dequeue; each adds
// 1 to the count and its value to the sum; a request's reply is (count after
// it, value).
__device__ __noinline__ void run_sink(const DrainParams &P, uint32_t a) {
    const uint32_t lane = lane_id();
    ActorDesc *A = &P.actors[a];
    if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
    __syncwarp();
    uint64_t head = *((volatile uint64_t *)&A->head);
    const uint64_t tail = ld_acquire_gpu(&A->tail);
    uint64_t left = tail - head;
    if (left > kSinkChunk) left = kSinkChunk;
    // tail counts tickets a sender may not have published yet; a ticket at or
    // past head + capacity waits for room that this claim only releases at
    // its end, so a claim never goes past one mailbox's worth
    if (left > (uint64_t)A->cap_mask + 1) left = (uint64_t)A->cap_mask + 1;
    if (P.max_claim && left > P.max_claim) left = P.max_claim;
    if (lane == 0) add_u64(&P.ctl->claims, 1);
    uint64_t count = A->sink_count, sum = A->sink_sum, handled = 0;
    while (left > 0) {
        // up to 128 messages per round of loads (the 32-wide dequeue in
        // validation mode, for its log, and to wait for an unpublished head)
        if (!P.validation && left > 32) {
            uint64_t v = 0;
            const uint32_t got = sink_take_wide(P, a, head, left < 128 ? (uint32_t)left : 128u, count, &v);
            if (got > 0) {   // handled (replies written): 0 only when head is unpublished
                sum += warp_sum_u64(v);
                count += got;
                handled += got;
                head += got;
                left -= got;
                continue;
            }
        }
        MsgData m{};
        const uint32_t got = warp_dequeue(P, a, head, left < 32 ? (uint32_t)left : 32u, m);
        if (got == 0) break;
        const uint64_t v = lane < got ? m.payload : 0;
        if (lane < got) write_reply(m.reply_addr, 0, count + lane + 1, v, m.tag, m.reply_token);
        sum += warp_sum_u64(v);
        count += got;
        handled += got;
        head += got;
        left -= got;
    }
    if (lane == 0) {
        A->sink_count = count;
        A->sink_sum = sum;
        __threadfence();
        add_u64(&P.ctl->messages, handled);
        add_u64(&P.ctl->completed, handled);
    }
    __syncwarp();
    release_actor(P, a, head);
}

// Claimed SOURCE `a`: handle one message, (c remaining, k0 first index) with
// c in the low and k0 in the high 32 bits: send up to kSourceChunk messages
// (k0 + i) to the target SINK, 32 per warp-wide enqueue, then either send the
// continuation (c', k0') to itself or, when all are sent, reply (total, 0).
__device__ __noinline__ void run_source(const DrainParams &P, uint32_t a) {
    const uint32_t lane = lane_id();
    ActorDesc *A = &P.actors[a];
    if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
    __syncwarp();
    const uint64_t head = *((volatile uint64_t *)&A->head);
    if (lane == 0) add_u64(&P.ctl->claims, 1);
    MsgData m{};
    if (warp_dequeue(P, a, head, 1, m) == 0) return;
    m.payload = __shfl_sync(FULL, m.payload, 0);
    m.reply_addr = __shfl_sync(FULL, m.reply_addr, 0);
    m.reply_token = __shfl_sync(FULL, m.reply_token, 0);
    m.tag = __shfl_sync(FULL, m.tag, 0);
    const uint32_t c = (uint32_t)m.payload, k0 = (uint32_t)(m.payload >> 32);
    const uint32_t now = c < kSourceChunk ? c : kSourceChunk;
    const uint32_t target = A->next;
    bool ok = true;
    for (uint32_t i = 0; i < now && ok; i += 32) {
        MsgData s{};
        const uint32_t k = k0 + i + lane;
        s.payload = ((uint64_t)a << 32) | k;
        s.kind = kSink;
        s.sender = 0x80000000u | a;
        s.sender_seq = k;
        s.tag = k;
        ok = warp_enqueue(P, i + lane < now, target, s);
    }
    if (lane == 0) add_u64(&P.ctl->device_sends, now);
    if (ok && now < c) {
        MsgData s = m;   // continuation: same reply route
        s.payload = ((uint64_t)(k0 + now) << 32) | (c - now);
        s.kind = kSource;
        s.sender = 0x80000000u | a;
        s.sender_seq = k0 + now;
        ok = warp_enqueue(P, lane == 0, a, s);
    } else if (ok && lane == 0) {
        write_reply(m.reply_addr, 0, k0 + now, 0, m.tag, m.reply_token);
    }
    if (lane == 0) {
        __threadfence();
        add_u64(&P.ctl->messages, 1);
        add_u64(&P.ctl->completed, 1);
    }
    __syncwarp();
    release_actor(P, a, head + 1);
}

// ---------------------------------------------------------------------------
// FORK actors: recursive actor creation (Sec. 5, "Overhead of Actor
// Creation": 2^n computed by actors that each spawn two actors with counter
// n - 1 and wait for their results).  Spawned actors come from a device pool
// of actor ids with fixed 4-slot mailboxes; an actor that has answered
// terminates and its id goes back to the pool, so repeated computations
// recycle the same records.  A result message carries the child's value in
// its low and the actors spawned below it in its high 32 bits.
// ---------------------------------------------------------------------------
// Lane 0: take a free pool id, waiting (bounded) while the pool is empty.
__device__ uint32_t fork_take_id(const DrainParams &P) {
    uint32_t id = kNone;
    WaitClock w(P.wait_limit_ns);
    for (;;) {
        const int pr = q_try_pop(&P.ctl->forkq, P.forkq, &id, P.wait_limit_ns);
        if (pr > 0) return id;
        if (pr < 0 || !w.again()) {
            fail(P, kErrWaitQueue, 29, 0, 0);
            return kNone;
        }
        __nanosleep(64);
    }
}

// Answer (value, spawned below) to the parent, or to the root's requester.
__device__ bool fork_answer(const DrainParams &P, uint32_t a, uint64_t value, uint64_t spawned) {
    ActorDesc *A = &P.actors[a];
    const uint32_t parent = A->next;
    if (parent == kNone) {
        if (lane_id() == 0) write_reply(A->fork_reply, 0, value, spawned, 0, A->fork_token);
        __syncwarp();
        return true;
    }
    MsgData r{};
    r.payload = (value & 0xFFFFFFFFull) | (spawned << 32);
    r.kind = kFork | (kMsgResult << 16);
    r.sender = 0x80000000u | a;
    if (lane_id() == 0) add_u64(&P.ctl->device_sends, 1);
    return warp_enqueue(P, lane_id() == 0, parent, r);
}

// Claimed FORK actor `a`: handle its published messages in mailbox order.  A
// start message with counter c answers 1 when c = 0; otherwise it spawns two
// pool actors (parent a, counter c - 1) and sends each a start message.  A
// result adds to the actor's sum; the second one answers (sum, 2 + spawned
// below).  A pool actor terminates after answering and returns its id to the
// pool; a root (spawned by the host) stays for the next computation.  A start
// message that reaches a root still waiting for results is rejected.
__device__ __noinline__ void run_fork(const DrainParams &P, uint32_t a) {
    const uint32_t lane = lane_id();
    ActorDesc *A = &P.actors[a];
    const bool pooled = a >= P.fork_base && a - P.fork_base < P.fork_pool;
    if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
    __syncwarp();
    const uint64_t head = *((volatile uint64_t *)&A->head);
    const uint64_t tail = ld_acquire_gpu(&A->tail);
    uint64_t avail = tail - head;
    if (P.max_claim && avail > P.max_claim) avail = P.max_claim;
    if (lane == 0) add_u64(&P.ctl->claims, 1);
    MsgData m{};
    const uint32_t got = avail ? warp_dequeue(P, a, head, avail < 32 ? (uint32_t)avail : 32u, m) : 0u;
    int32_t pending = A->user_state;
    uint64_t sum = A->sink_sum, spawned = A->sink_count;
    bool ok = true, ended = false;
    for (uint32_t i = 0; i < got && ok; ++i) {
        const uint64_t v = __shfl_sync(FULL, m.payload, i);
        const uint32_t kind = __shfl_sync(FULL, m.kind, i);
        const uint64_t reply_addr = __shfl_sync(FULL, m.reply_addr, i);
        const uint32_t token = __shfl_sync(FULL, m.reply_token, i);
        const uint64_t tag = __shfl_sync(FULL, m.tag, i);
        if (!((kind >> 16) & kMsgResult)) {
            if (pending != 0 || ended) {
                if (lane == 0) write_reply(reply_addr, 3, 0, 0, tag, token);
                continue;
            }
            if (!pooled && lane == 0) {
                A->fork_reply = reply_addr;
                A->fork_token = token;
            }
            __syncwarp();
            if (v == 0) {
                ok = fork_answer(P, a, 1, 0);
                ended = pooled;          // a root takes its next start message
                continue;
            }
            // spawn two children: lanes 0 and 1 each take a pool id and set it up
            uint32_t c = kNone;
            if (lane < 2) {
                c = fork_take_id(P);
                if (c != kNone) {
                    ActorDesc *C = &P.actors[c];
                    C->kind = kFork;      // the record may have served a ring member
                    C->flags = 0;
                    C->next = a;
                    C->user_state = 0;
                    C->sink_sum = 0;
                    C->sink_count = 0;
                    C->fork_reply = 0;
                    *((volatile uint32_t *)&C->state) = kWaiting;
                }
            }
            if (__any_sync(FULL, lane < 2 && c == kNone)) {
                ok = false;
                break;
            }
            __threadfence();
            MsgData s{};
            s.payload = v - 1;
            s.kind = kFork;
            s.sender = 0x80000000u | a;
            s.sender_seq = lane;
            s.tag = tag;
            if (lane == 0) {
                add_u64(&P.ctl->device_sends, 2);
                add_u64(&P.ctl->device_spawns, 2);
            }
            ok = warp_enqueue(P, lane < 2, c, s);
            pending = 2;
            sum = 0;
            spawned = 0;
        } else {
            sum += v & 0xFFFFFFFFull;
            spawned += v >> 32;
            if (--pending == 0) {
                ok = fork_answer(P, a, sum, spawned + 2);
                ended = pooled;
                sum = 0;
                spawned = 0;
            }
        }
    }
    if (lane == 0) {
        if (ended) {
            // a pool actor that has answered terminates
            A->user_state = 0;
            A->sink_sum = 0;
            A->sink_count = 0;
            *((volatile uint32_t *)&A->state) = kDone;
        } else {
            A->user_state = pending;
            A->sink_sum = sum;
            A->sink_count = spawned;
        }
        __threadfence();
        add_u64(&P.ctl->messages, got);
        add_u64(&P.ctl->completed, got);
    }
    __syncwarp();
    release_actor(P, a, head + got);
    if (ended && pooled && lane == 0) {
        // every message of this incarnation is handled and the claim is
        // released: the id can serve a new actor
        __threadfence();
        if (!q_push(&P.ctl->forkq, P.forkq, a, P.wait_limit_ns)) fail(P, kErrWaitQueue, 30);
    }
    __syncwarp();
}

// Answer a message that cannot be handled (unknown actor, kind mismatch,
// terminated receiver, n out of range).
__device__ __forceinline__ void reject(uint64_t reply_addr, uint32_t token, uint64_t tag, int32_t status) {
    write_reply(reply_addr, status, 0, 0, tag, token);
}

__device__ __forceinline__ bool message_ok(const DrainParams &P, uint32_t a, uint32_t kind, uint64_t payload,
                                           int32_t *why) {
    if (a >= P.n_actors) { *why = 3; return false; }
    const ActorDesc *A = &P.actors[a];
    if ((kind & 0xFFFFu) != A->kind) { *why = 3; return false; }
    if (*((volatile const uint32_t *)&A->state) == kDone) { *why = 2; return false; }
    if ((kind & 0xFFFFu) == kFactor && payload > P.max_n) { *why = 3; return false; }
    // a token is a 31-bit value; the end-of-incarnation notice comes only from the device
    if ((kind & 0xFFFFu) == kToken && (payload > 0x7FFFFFFFull || ((kind >> 16) & kMsgRingDone))) {
        *why = 3;
        return false;
    }
    if ((kind & 0xFFFFu) == kFork) {
        // a start message whose tree fits the pool; results come only from children
        if (((kind >> 16) & kMsgResult) || payload > kForkMaxN || (2ull << payload) - 2 > P.fork_pool) {
            *why = 3;
            return false;
        }
    }
    return true;
}

// Device batch routing: router r takes the messages whose actor id is r
// modulo the router count, scanning the batch in array order, so each
// actor's messages enter its mailbox in array order.
__device__ void route_batch(const DrainParams &P, uint32_t r) {
    const uint32_t lane = lane_id();
    const caf_dmsg_t *msgs = reinterpret_cast<const caf_dmsg_t *>(P.batch_msgs);
    for (uint32_t base = 0; base < P.batch_count; base += 32) {
        const uint32_t i = base + lane;
        bool mine = false;
        caf_dmsg_t d{};
        if (i < P.batch_count) {
            d = msgs[i];
            mine = (d.actor % P.n_routers) == r;
        }
        if (!__any_sync(FULL, mine)) continue;
        int32_t why = 0;
        const bool ok = mine && message_ok(P, d.actor, d.kind, d.u64, &why);
        Reply *rep = P.batch_replies ? &P.batch_replies[i] : nullptr;
        if (mine && !ok) reject((uint64_t)rep, 1, d.tag, why);
        MsgData m{};
        m.payload = d.u64;
        m.reply_addr = (uint64_t)rep;
        m.reply_token = 1;
        m.tag = d.tag;
        m.sender = d.sender;
        m.sender_seq = d.sender_seq;
        m.kind = d.kind;
        if (!warp_enqueue(P, ok, d.actor, m)) return;
        if ((base & 4095u) == 0 && lane == 0) heartbeat(P);
    }
}

// Live ingress: take the published prefix of the host ring (in ticket order)
// and route it.  Returns true if anything was taken.
__device__ bool poll_host_ring(const DrainParams &P) {
    const uint32_t lane = lane_id();
    const uint64_t head = P.ctl->ring_head;
    IngressEntry *e = &P.ring[(head + lane) & P.ring_mask];
    const bool pub = ld_acquire_sys(&e->seq) == head + lane + 1;
    const uint32_t pm = __ballot_sync(FULL, pub);
    const uint32_t n = (pm == FULL) ? 32u : (uint32_t)(__ffs(~pm) - 1);
    if (n == 0) return false;
    const bool take = lane < n;
    MsgData m{};
    uint32_t a = 0;
    if (take) {
        a = e->actor;
        m.payload = e->payload;
        m.reply_addr = e->reply_addr;
        m.tag = e->tag;
        m.sender = e->sender;
        m.sender_seq = e->sender_seq;
        m.kind = e->kind;
        m.reply_token = e->reply_token;
    }
    int32_t why = 0;
    const bool ok = take && message_ok(P, a, m.kind, m.payload, &why);
    if (take && !ok) reject(m.reply_addr, m.reply_token, m.tag, why);
    if (!warp_enqueue(P, ok, a, m)) return true;
    if (lane == 0) {
        P.ctl->ring_head = head + n;
        st_release_sys(&P.hctl->ring_consumed, head + n);
    }
    __syncwarp();
    return true;
}

__device__ __forceinline__ bool quiescent(const DrainParams &P) {
    if (P.batch_count && *((volatile uint32_t *)&P.ctl->routers_done) < P.n_routers) return false;
    const uint64_t c = ld_acquire_gpu(&P.ctl->completed);
    const uint64_t i = ld_acquire_gpu(&P.ctl->ingested);
    return c == i;
}

// ---------------------------------------------------------------------------
// GEMM actors in the drain
// ---------------------------------------------------------------------------
// Warp-collective push of `count` items base | i (i < count) into an MPMC
// queue, positions reserved with one atomic add.
__device__ bool q_push_block(const DrainParams &P, QueueHdr *q, QCell *cells, uint32_t base, uint32_t count) {
    const uint32_t lane = lane_id();
    uint64_t pos0 = 0;
    if (lane == 0) pos0 = add_u64(&q->enq, count);
    pos0 = __shfl_sync(FULL, pos0, 0);
    bool ok = true;
    for (uint32_t i = lane; i < count && ok; i += 32) {
        const uint64_t pos = pos0 + i;
        QCell *c = &cells[pos & q->mask];
        if (ld_acquire_gpu(&c->seq) != pos) {
            WaitClock w(P.wait_limit_ns);
            while (ld_acquire_gpu(&c->seq) != pos) {
                if (!w.again()) { ok = false; break; }
            }
        }
        if (ok) {
            c->val = base | i;
            st_release_gpu(&c->seq, pos + 1);
        }
    }
    if (!__all_sync(FULL, ok)) {
        if (lane == 0) fail(P, kErrWaitQueue, 15, count, base);
        return false;
    }
    if (lane == 0) q_avail_add(q, count);
    return true;
}

// Warp-collective push of a run of items per lane: lane i pushes base_i | k
// for k < count_i, lanes in lane order, all positions reserved with one
// atomic add.  Position idx of the total belongs to the largest lane whose
// exclusive prefix is <= idx (found by a binary search over the lanes).
__device__ bool q_push_runs(const DrainParams &P, QueueHdr *q, QCell *cells, uint32_t base, uint32_t count) {
    const uint32_t lane = lane_id();
    uint32_t incl = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(FULL, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    const uint32_t excl = incl - count;
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0) return true;
    uint64_t pos0 = 0;
    if (lane == 0) pos0 = add_u64(&q->enq, total);
    pos0 = __shfl_sync(FULL, pos0, 0);
    bool ok = true;
    for (uint32_t at = 0; at < total; at += 32) {
        const uint32_t idx = at + lane;
        uint32_t o = 0;
#pragma unroll
        for (uint32_t step = 16; step; step >>= 1) {
            const uint32_t cand = o + step;
            const uint32_t e = __shfl_sync(FULL, excl, cand & 31u);
            if (cand < 32 && e <= idx) o = cand;
        }
        const uint32_t ob = __shfl_sync(FULL, base, o);
        const uint32_t oe = __shfl_sync(FULL, excl, o);
        if (idx < total && ok) {
            const uint64_t pos = pos0 + idx;
            QCell *c = &cells[pos & q->mask];
            if (ld_acquire_gpu(&c->seq) != pos) {
                WaitClock w(P.wait_limit_ns);
                while (ld_acquire_gpu(&c->seq) != pos) {
                    if (!w.again()) { ok = false; break; }
                }
            }
            if (ok) {
                c->val = ob | (idx - oe);
                st_release_gpu(&c->seq, pos + 1);
            }
        }
    }
    if (!__all_sync(FULL, ok)) {
        if (lane == 0) fail(P, kErrWaitQueue, 28, total, base);
        return false;
    }
    if (lane == 0) q_avail_add(q, total);
    return true;
}

// Job record j's queue and packed-operand scratch.
__device__ __forceinline__ bool job_small(uint32_t j) { return j < kGemmJobsSmall; }
__device__ __forceinline__ uint8_t *job_scratch(const DrainParams &P, uint32_t j) {
    return job_small(j) ? P.pack_small + (size_t)j * kPackSmallBytes
                        : P.pack_large + (size_t)(j - kGemmJobsSmall) * kPackLargeBytes;
}
__device__ __forceinline__ bool job_free(const DrainParams &P, uint32_t j) {
    return job_small(j) ? q_push(&P.ctl->jobq, P.jobq, j, P.wait_limit_ns)
                        : q_push(&P.ctl->jobq_large, P.jobq_large, j, P.wait_limit_ns);
}

// Read the job fields of tile item `item` (job << 16 | tile index) into `s`
// and check them: a record inside the table, a size its scratch class holds,
// the tile count the size gives, and a tile index below it (so the tile lies
// inside the matrix and its images inside the record's scratch).  The
// images' address comes from the record index, not from the record.
__device__ __forceinline__ bool tile_snap(const DrainParams &P, uint32_t item, TileSnap &s) {
    const uint32_t j = item >> 16, idx = item & 0xFFFFu;
    s = TileSnap{};
    if (j >= kGemmJobs) return false;
    const GemmJob *J = &P.jobs[j];
    const uint32_t n = J->n, flags = J->split, tiles = J->tiles;
    const uint64_t C = J->C;
    s.tiles = tiles;
    if (n == 0 || n > (job_small(j) ? kPackSmallMaxN : kMaxDrainGemmN) || flags > 3u) return false;
    const uint32_t t = (n + kGemmBN - 1) / kGemmBN, tw = (flags & 2u) ? (t + 1) / 2 : t;
    if (tiles != t * tw || idx >= tiles || (flags & 3u) == 3u) return false;
    s.pack = reinterpret_cast<uint64_t>(job_scratch(P, j));
    s.C = C;
    s.n = n;
    s.split = (uint8_t)(flags & 1u);
    s.tm = (uint16_t)(idx / tw);
    s.tn = (uint16_t)((flags & 2u) ? 2 * (idx % tw) : idx % tw);
    s.wide = (uint8_t)((flags & 2u) && s.tn + 1u < t);
    return true;
}

__device__ bool work_item_ok(const DrainParams &P, uint32_t item) {
    const uint32_t j = item >> 16;
    if (item & kPackItemFlag) {
        if (j >= kGemmJobs) return false;
        return (item & 63u) < (P.jobs[j].n + kGemmBN - 1) / kGemmBN;
    }
    if (item & kMandelItemFlag) return j < kMandelJobs && (item & (kMandelItemFlag - 1u)) < P.mjobs[j].bands;
    return j < kGemmJobs && (item & 0xFFFFu) < P.jobs[j].tiles;
}

// Claim a GEMM actor: take up to 32 messages (as many as there are free job
// records of the size class each needs), turn each into a job and queue its
// pack items (two per 128-wide panel: one of A, one of B^T).
__device__ __noinline__ void claim_gemm(const DrainParams &P, uint32_t a) {
    const uint32_t lane = lane_id();
    DevCtl *ctl = P.ctl;
    ActorDesc *A = &P.actors[a];
    const uint32_t split = A->kind == kGemmSplit ? 1u : 0u;
    if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
    __syncwarp();
    const uint64_t head = *((volatile uint64_t *)&A->head);
    const uint64_t tail = ld_acquire_gpu(&A->tail);
    uint64_t avail = tail - head;
    // (the runtime's per-claim message limit is not applied here: GEMM
    // claims of at most 8 messages with 128 x 256 tiles faulted the GPU, for
    // a cause not yet found)
    const uint32_t want = avail < 32 ? (uint32_t)avail : 32u;
    if (lane == 0) add_u64(&ctl->claims, 1);
    // read each message's descriptor in place (published slots only), then
    // reserve a job record of its class, so a claim never waits for one
    const uint64_t t = head + lane;
    const Slot *sl = &P.slots[A->slot_base + (t & A->cap_mask)];
    const bool pub = lane < want && ld_acquire_gpu(&sl->seq) == t + 1;
    const uint32_t pm = __ballot_sync(FULL, pub);
    const uint32_t npub = (pm == FULL) ? 32u : (uint32_t)(__ffs(~pm) - 1);
    const GemmDesc *d = lane < npub ? reinterpret_cast<const GemmDesc *>(sl->payload) : nullptr;
    const uint32_t n = d ? d->n : 0u;
    // (a drain launched without packed-operand scratch rejects GEMM messages)
    const bool valid = d && n > 0 && n <= kMaxDrainGemmN && d->A && d->B && d->C && P.pack_small && P.pack_large;
    uint32_t j = kNone;
    bool got = false;
    if (valid) {
        const int pr = n <= kPackSmallMaxN ? q_try_pop(&ctl->jobq, P.jobq, &j, P.wait_limit_ns)
                                           : q_try_pop(&ctl->jobq_large, P.jobq_large, &j, P.wait_limit_ns);
        if (pr < 0) fail(P, kErrWaitQueue, 21);
        got = pr > 0;
    }
    const uint32_t okm = __ballot_sync(FULL, lane < npub && (!valid || got));
    const uint32_t nj = (okm == FULL) ? 32u : (uint32_t)(__ffs(~okm) - 1);
    MsgData m{};
    const uint32_t take = nj ? warp_dequeue(P, a, head, nj, m) : 0u;
    if (got && lane >= take) {
        job_free(P, j);
        got = false;
    }
    release_actor(P, a, head + take);
    uint32_t panels = 0;
    if (lane < take) {
        if (valid) {
            const uint32_t tt = (n + kGemmBN - 1) / kGemmBN;
            // BF16 jobs run wide tiles: 128 rows x 256 columns (two B panels)
            // per item, a narrow one for the last column of an odd panel count
            const bool wide = !split && P.gemm_wide;
            GemmJob *J = &P.jobs[j];
            J->A = d->A;
            J->B = d->B;
            J->C = d->C;
            J->n = n;
            J->split = split | (wide ? 2u : 0u);
            J->tiles = wide ? tt * ((tt + 1) / 2) : tt * tt;
            J->done = 0;
            J->packs_left = 2 * tt;
            J->reply_addr = m.reply_addr;
            J->reply_token = m.reply_token;
            panels = tt;
        } else {
            write_reply(m.reply_addr, 3, 0, n, m.tag, m.reply_token);
        }
    }
    const uint32_t bad = __popc(__ballot_sync(FULL, lane < take && !valid));
    if (lane == 0 && bad) {
        __threadfence();
        add_u64(&ctl->completed, bad);
    }
    __threadfence();
    for (uint32_t i = 0; i < take; ++i) {
        const uint32_t pi = __shfl_sync(FULL, panels, i);
        const uint32_t ji = __shfl_sync(FULL, j, i);
        if (!pi) continue;
        if (!q_push_block(P, &ctl->packq, P.packq, (ji << 16) | kPackItemFlag, pi)) return;
        if (!q_push_block(P, &ctl->packq, P.packq, (ji << 16) | kPackItemFlag | 64u, pi)) return;
    }
}

struct NamedBarSync {
    uint32_t nthreads;
    __device__ __forceinline__ void operator()() const { named_bar_sync(1, nthreads); }
};

// Run GEMM pack item `item` (flag kPackItemFlag; bit 6: B instead of A; bits
// 0..5: panel) with the whole CTA; the CTA that finishes a job's last pack
// item queues its tiles.
__device__ __noinline__ void drain_gemm_pack(const DrainParams &P, PackedSlots &slots, uint32_t item,
                                             uint32_t bar_threads) {
    const uint32_t j = item >> 16, x = item & 0xFFFFu;
    GemmJob *J = &P.jobs[j];
    const uint32_t n = J->n;
    const bool split = (J->split & 1u) != 0;
    const PackGeom g = pack_geom(job_scratch(P, j), n, split);
    const uint32_t panel = x & 63u;
    if ((threadIdx.x >> 5) < kGemmConvWarps) {
        const float *src = reinterpret_cast<const float *>((x & 64u) ? J->B : J->A);
        // staged copies need 16-byte aligned rows
        const bool staged = (n & 3u) == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
        uint8_t *stage = reinterpret_cast<uint8_t *>(&slots);
        if (x & 64u) {
            if (staged) gemm_pack_b_staged(src, g, panel, split, stage);
            else gemm_pack_b(src, g, panel, split);
        } else {
            if (staged) gemm_pack_a_staged(src, g, panel, split, stage);
            else gemm_pack_a(src, g, panel, split);
        }
    }
    named_bar_sync(1, bar_threads);
    if (threadIdx.x < 32) {
        uint32_t last = 0;
        if (threadIdx.x == 0) {
            heartbeat(P);
            __threadfence();   // this CTA's packed stores before the count
            last = atomicSub(reinterpret_cast<unsigned int *>(&J->packs_left), 1u) == 1u;
        }
        if (__shfl_sync(FULL, last, 0)) {
            __threadfence();
            if (!q_push_block(P, &P.ctl->workq, P.workq, j << 16, J->tiles) && threadIdx.x == 0)
                fail(P, kErrWaitQueue, 18);
        }
    }
}

// Tile i of a run of tile items, from the snapshots taken with the items.
struct RunTile {
    const TileSnap *snap;
    __device__ TileRef operator()(uint32_t i) const {
        const TileSnap &s = snap[i];
        TileRef r;
        r.split = s.split != 0;
        r.wide = s.wide != 0;
        r.g = pack_geom(reinterpret_cast<uint8_t *>(s.pack), s.n, r.split);
        r.C = reinterpret_cast<float *>(s.C);
        r.tm = s.tm;
        r.tn = s.tn;
        return r;
    }
};

// Run `count` tile items (their snapshots: `snap`) as one pipeline with the
// whole CTA; for each, the CTA that finishes a job's last tile writes its
// reply and frees the record.
__device__ __noinline__ void drain_gemm_tiles(const DrainParams &P, GroupShared &G, PackedSlots &slots,
                                              const uint32_t *items, const TileSnap *snap, uint32_t count,
                                              GemmCounters &K, uint32_t bar_threads) {
    // `items` and `snap` are shared memory the producer warp refills for its
    // next round once the sequence's last barrier has passed: keep this run's
    // ids and counts
    uint32_t mine[kMaxItemsPerRound], tiles_of[kMaxItemsPerRound];
    uint32_t equiv = 0;   // 128 x 128 output tiles these items cover
    if (threadIdx.x == 0) {
#pragma unroll
        for (uint32_t i = 0; i < kMaxItemsPerRound; ++i) {
            mine[i] = i < count ? items[i] : 0u;
            tiles_of[i] = i < count ? snap[i].tiles : 0u;
            equiv += i < count ? (snap[i].wide ? 2u : 1u) : 0u;
        }
    }
    const bool ok = gemm_tiles_packed(RunTile{snap}, count, slots, G.gb, K, P.wait_limit_ns,
                                      NamedBarSync{bar_threads});
    items = nullptr;
    snap = nullptr;
    if (threadIdx.x == 0) {
        if (!ok) fail(P, kErrGemm, 16, mine[0], count);
        heartbeat(P);
        __threadfence();
        add_u64(&P.ctl->gemm_tiles, equiv);
#pragma unroll
        for (uint32_t i = 0; i < kMaxItemsPerRound; ++i) {
            if (i >= count) break;
            const uint32_t j = mine[i] >> 16;
            GemmJob *J = &P.jobs[j];
            // the tile count was read before this CTA counted its tile: the
            // record cannot have been freed and reused in between
            const uint32_t before = atomicAdd(reinterpret_cast<unsigned int *>(&J->done), 1u);
            if (before >= tiles_of[i]) {
                fail(P, kErrGemm, 19, mine[i], before);   // a tile counted twice
            } else if (before + 1u == tiles_of[i]) {
                __threadfence();
                write_reply(J->reply_addr, ok ? 0 : 3, 0, J->n, 0, J->reply_token);
                __threadfence();
                add_u64(&P.ctl->messages, 1);
                add_u64(&P.ctl->completed, 1);
                if (!job_free(P, j)) fail(P, kErrWaitQueue, 17);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Mandelbrot actors in the drain
// ---------------------------------------------------------------------------
// Claim a Mandelbrot actor: take up to 32 messages (as many as there are free
// job records), copy each message's descriptor into its job and queue the
// job's bands as work items.  The claim's jobs together are cut into about
// two bands per CTA of the grid, in proportion to their pixels, so a single
// large image fills every SM; bands stay within [kMandelBandMin,
// kMandelBandMax] pixels (large bands when the claim brings plenty of work:
// each band costs a round's pop, barrier and count update).
__device__ __noinline__ void claim_mandel(const DrainParams &P, uint32_t a) {
    const uint32_t lane = lane_id();
    DevCtl *ctl = P.ctl;
    ActorDesc *A = &P.actors[a];
    if (lane == 0) *((volatile uint32_t *)&A->state) = kRunning;
    __syncwarp();
    const uint64_t head = *((volatile uint64_t *)&A->head);
    const uint64_t tail = ld_acquire_gpu(&A->tail);
    const uint64_t avail = tail - head;
    uint32_t want = avail < 32 ? (uint32_t)avail : 32u;
    if (P.max_claim && P.max_claim < want) want = P.max_claim;
    if (lane == 0) add_u64(&ctl->claims, 1);
    // a record per message, reserved before the dequeue so a claim never waits for one
    uint32_t j = kNone;
    bool got = false;
    if (lane < want) {
        const int pr = q_try_pop(&ctl->mjobq, P.mjobq, &j, P.wait_limit_ns);
        if (pr < 0) fail(P, kErrWaitQueue, 25);
        got = pr > 0;
    }
    const uint32_t okm = __ballot_sync(FULL, got);
    const uint32_t nj = (okm == FULL) ? 32u : (uint32_t)(__ffs(~okm) - 1);
    MsgData m{};
    const uint32_t take = nj ? warp_dequeue(P, a, head, nj, m) : 0u;
    if (got && lane >= take) {
        if (!q_push(&ctl->mjobq, P.mjobq, j, P.wait_limit_ns)) fail(P, kErrWaitQueue, 26);
        got = false;
    }
    release_actor(P, a, head + take);
    uint32_t bands = 0;
    bool valid = false;
    MandelDesc d{};
    if (lane < take) {
        const MandelDesc *dp = reinterpret_cast<const MandelDesc *>(m.payload);
        if (dp) d = *dp;
        valid = dp && mandel_desc_ok(d);
    }
    const uint64_t claim_px = warp_sum_u64(valid ? (uint64_t)d.width * d.rows : 0ull);
    if (lane < take) {
        if (valid) {
            MandelJob *J = &P.mjobs[j];
            J->d = d;
            const uint32_t pixels = d.width * d.rows;
            const uint64_t tq = (2ull * gridDim.x * pixels + claim_px - 1) / claim_px;
            const uint32_t target = tq < kMandelMaxBands ? (uint32_t)tq : kMandelMaxBands;
            const uint32_t nb = max((pixels + kMandelBandMax - 1) / kMandelBandMax,
                                    min((pixels + kMandelBandMin - 1) / kMandelBandMin, target));
            const uint32_t band_px = ((pixels + nb - 1) / nb + 31u) & ~31u;
            bands = (pixels + band_px - 1) / band_px;
            J->band_px = band_px;
            J->bands = bands;
            J->done = 0;
            J->sum = 0;
            J->reply_addr = m.reply_addr;
            J->reply_token = m.reply_token;
        } else {
            write_reply(m.reply_addr, 3, 0, 0, m.tag, m.reply_token);
            if (!q_push(&ctl->mjobq, P.mjobq, j, P.wait_limit_ns)) fail(P, kErrWaitQueue, 26);
        }
    }
    const uint32_t bad = __popc(__ballot_sync(FULL, lane < take && !valid));
    if (lane == 0 && bad) {
        __threadfence();
        add_u64(&ctl->completed, bad);
    }
    __threadfence();
    q_push_runs(P, &ctl->workq, P.workq, (j << 16) | kMandelItemFlag, bands);
}

// Entry i of a small register array (no dynamic indexing, so no local memory).
template <uint32_t N>
__device__ __forceinline__ uint32_t pick_item(const uint32_t (&a)[N], uint32_t i) {
    uint32_t v = a[0];
#pragma unroll
    for (uint32_t k = 1; k < N; ++k)
        if (k == i) v = a[k];
    return v;
}

// Run `count` Mandelbrot band items with the whole CTA as one pool of 32-pixel
// groups: each warp takes the next group from a shared counter (so slow and
// fast regions even out), lane l computes pixel 32 g + l of its band.  Then,
// per band, thread 0 adds the band's count sum to its job, and the CTA that
// finishes a job's last band writes the reply (pixels, sum of the counts) and
// frees the record.  G.mnext and G.msum are zero on entry; thread 0 zeroes them
// again after the closing barrier, before it reaches the next round's.
__device__ __noinline__ void drain_mandel_bands(const DrainParams &P, GroupShared &G, const uint32_t *items,
                                                uint32_t count, uint32_t bar_threads) {
    const uint32_t lane = lane_id();
    uint32_t mine[kMaxItemsPerRound];
    uint32_t first[kMaxItemsPerRound + 1];     // first group of each band in the pool
    first[0] = 0;
#pragma unroll
    for (uint32_t i = 0; i < kMaxItemsPerRound; ++i) {
        mine[i] = i < count ? items[i] : 0u;
        const uint32_t groups = i < count ? P.mjobs[mine[i] >> 16].band_px / 32u : 0u;
        first[i + 1] = first[i] + groups;
    }
    const uint32_t total = first[kMaxItemsPerRound];
    uint32_t cur = kNone;                  // band whose descriptor is in registers
    uint32_t base = 0, gbase = 0;          // its first pixel and first group
    MandelDesc d{};
    uint32_t pixels = 0;
    unsigned long long acc = 0;            // this lane's count sum for band `cur`
    for (;;) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(&G.mnext, 1u);
        g = __shfl_sync(FULL, g, 0);
        uint32_t b = kNone;
        if (g < total) {
            b = 0;
#pragma unroll
            for (uint32_t i = 1; i < kMaxItemsPerRound; ++i)
                if (g >= first[i]) b = i;
        }
        // (a warp whose first group is already past the pool's end leaves
        // too: cur is still kNone then)
        if (b != cur || b == kNone) {
            if (cur != kNone) {
                const unsigned long long s = warp_sum_u64(acc);
                if (lane == 0 && s) atomicAdd(&G.msum[cur], s);
            }
            acc = 0;
            cur = b;
            if (b == kNone) break;
            const uint32_t it = pick_item(mine, b);
            const MandelJob *J = &P.mjobs[it >> 16];
            d = J->d;
            pixels = d.width * d.rows;
            base = (it & (kMandelItemFlag - 1u)) * J->band_px;
            gbase = pick_item(first, b);
        }
        // long bands (max_iter up to 65536) keep the stall detector fed
        if (lane == 0 && (g & 15u) == 0) heartbeat(P);
        const uint32_t p = base + (g - gbase) * 32u + lane;
        if (p < pixels) {
            float cx, cy;
            mandel_c(d, p, cx, cy);
            const uint32_t k = mandel_count(cx, cy, d.max_iter);
            reinterpret_cast<uint32_t *>(d.out)[p] = k;
            acc += k;
        }
    }
    named_bar_sync(1, bar_threads);
    if (threadIdx.x == 0) {
        heartbeat(P);
        __threadfence();   // the CTA's pixel stores before the band counts
#pragma unroll
        for (uint32_t i = 0; i < kMaxItemsPerRound; ++i) {
            if (i >= count) break;
            const uint32_t j = mine[i] >> 16;
            MandelJob *J = &P.mjobs[j];
            atomicAdd(reinterpret_cast<unsigned long long *>(&J->sum), G.msum[i]);
            G.msum[i] = 0;
            __threadfence();
            if (atomicAdd(reinterpret_cast<unsigned int *>(&J->done), 1u) == J->bands - 1) {
                __threadfence();
                const uint64_t sum = atomicAdd(reinterpret_cast<unsigned long long *>(&J->sum), 0ull);
                write_reply(J->reply_addr, 0, (uint64_t)J->d.width * J->d.rows, sum, 0, J->reply_token);
                __threadfence();
                add_u64(&P.ctl->messages, 1);
                add_u64(&P.ctl->completed, 1);
                if (!q_push(&P.ctl->mjobq, P.mjobq, j, P.wait_limit_ns)) fail(P, kErrWaitQueue, 27);
            }
        }
        G.mnext = 0;
    }
}

// Claim factor actor `a` (popped from the ready queue, kind checked) into
// batch records.  While more actors are ready than teams are idle, the claim
// fills a group of up to kGroupRecords records: messages of `a`, then of up to
// kTopUpTries further ready factor actors, reordered by n (factor_group_sort).
// The caller's team sweeps the group's last batch (the largest n); the
// others go to the queue of batches waiting for a team.  Otherwise the claim
// fills one record from `a` alone.  With no record free the actor stays
// READY.  Returns the batch the caller's team sweeps, or kNone.
template <bool kSplit>
__device__ __noinline__ uint32_t claim_factor_group(const DrainParams &P, uint32_t a, uint32_t rng) {
    const uint32_t lane = lane_id();
    DevCtl *ctl = P.ctl;
    const uint32_t K = P.factor_k;
    bool topup = false;
    if (lane == 0) {
        const int64_t teams = (int64_t)gridDim.x * (kConsumerWarps / P.factor_w);
        const int64_t busy = (int64_t)P.n_batches - q_len(&ctl->freeq);
        topup = q_len(&ctl->readyq) > teams - busy;
    }
    topup = __shfl_sync(FULL, topup, 0);
    const uint32_t want = topup ? min(kGroupRecords, kGroupMessages / K) : 1u;
    uint32_t b = kNone;
    bool gb = false;
    if (lane < want) {
        const int pr = q_try_pop(&ctl->freeq, P.freeq, &b, P.wait_limit_ns);
        if (pr < 0) fail(P, kErrWaitQueue, 23);
        gb = pr > 0;
        if (gb && P.validation && b >= P.n_batches) {
            bounds_fail(P, 44, b, P.n_batches);
            gb = false;
        }
    }
    const uint32_t gm = __ballot_sync(FULL, gb);
    if (gm == 0) {
        // no batch record free: leave the actor READY for later
        if (lane == 0 && !ready_push(P, a)) fail(P, kErrWaitQueue, 7);
        __syncwarp();
        return kNone;
    }
    // lane r < ng holds the group's record r (the records popped, in lane order)
    const uint32_t ng = __popc(gm);
    uint32_t m = gm;
    for (uint32_t i = 0; i < lane && i < ng; ++i) m &= m - 1;
    const uint32_t recs = __shfl_sync(FULL, b, lane < ng ? (uint32_t)(__ffs(m) - 1) : 0u);
    const uint32_t cap = ng * K;
    uint32_t count = claim_factor_take(P, a, recs, 0, cap);
    // top the group up with the messages of further ready factor actors (an
    // actor of another kind goes back to the ready queue)
    for (uint32_t extra = 0; topup && extra < kTopUpTries && count < cap; ++extra) {
        uint32_t a2 = 0;
        bool got2 = false;
        if (lane == 0) {
            const int pr = ready_pop(P, &a2, rng);
            if (pr < 0) fail(P, kErrWaitQueue, 36);
            got2 = pr > 0;
        }
        if (!__shfl_sync(FULL, got2, 0)) break;
        a2 = __shfl_sync(FULL, a2, 0);
        if (P.validation && !actor_ok(P, a2)) {
            if (lane == 0) bounds_fail(P, 46, a2, P.n_actors);
            break;
        }
        if (P.actors[a2].kind != kFactor) {
            if (lane == 0 && !ready_push(P, a2)) fail(P, kErrWaitQueue, 37);
            __syncwarp();
            break;
        }
        count = claim_factor_take(P, a2, recs, count, cap);
    }
    if (ng > 1 && count > K) factor_group_sort(P, recs, count);
    // launch each record; all but the last launched batch wait in the queue
    uint32_t mine = kNone;
    for (uint32_t r = 0; r < ng; ++r) {
        const uint32_t br = __shfl_sync(FULL, recs, r);
        const uint32_t cr = count > r * K ? min(count - r * K, K) : 0u;
        const uint32_t got = factor_batch_launch<kSplit>(P, br, cr);
        if (got == kNone) continue;
        if (mine != kNone) {
            // the record is complete before another team can take it
            __threadfence();
            bool ok = true;
            if (lane == 0) ok = q_push(&ctl->segq, P.segq, mine, P.wait_limit_ns);
            if (!__shfl_sync(FULL, ok, 0)) {
                if (lane == 0) fail(P, kErrWaitQueue, 38);
                return kNone;
            }
        }
        mine = got;
    }
    return mine;
}

// A team leader looks for a factor batch to sweep: a batch waiting in the
// queue first, else pop ready actors, claim factor actors into batch
// records, and run the other actors on the way (a few at most).
template <bool kGemm, bool kSplit>
__device__ uint32_t find_batch(const DrainParams &P, uint32_t &rng) {
    const uint32_t lane = lane_id();
    DevCtl *ctl = P.ctl;
    {
        // a batch (or a segment of a split batch) waiting for a team comes first
        uint32_t item = kNone;
        if (lane == 0) {
            const int pr = q_try_pop(&ctl->segq, P.segq, &item, P.wait_limit_ns);
            if (pr < 0) fail(P, kErrWaitQueue, 34);
            if (pr <= 0) item = kNone;
        }
        item = __shfl_sync(FULL, item, 0);
        if (item != kNone && P.validation && (item & 0xFFFFFFu) >= P.n_batches) {
            if (lane == 0) bounds_fail(P, 43, item, P.n_batches);
            return kNone;
        }
        if (item != kNone) return item;
    }
    for (int attempt = 0; attempt < 4; ++attempt) {
        uint32_t a = 0;
        bool got = false;
        if (lane == 0) {
            const int pr = ready_pop(P, &a, rng);
            if (pr < 0) fail(P, kErrWaitQueue, 22);
            got = pr > 0;
        }
        got = __shfl_sync(FULL, got, 0);
        if (!got) return kNone;
        a = __shfl_sync(FULL, a, 0);
        if (P.validation && !actor_ok(P, a)) {
            if (lane == 0) bounds_fail(P, 42, a, P.n_actors);
            return kNone;
        }
        const uint32_t kind = P.actors[a].kind;
        if (kind == kFactor) {
            // (the work-stealing scheduler's victim choice: a fresh draw here)
            const uint32_t r = claim_factor_group<kSplit>(P, a, rng);
            rng = rng * 1664525u + 1013904223u;
            if (r != kNone) return r;
        } else if (kind == kToken) {
            claim_ring(P, a);
        } else if (kind == kSink) {
            run_sink(P, a);
        } else if (kind == kSource) {
            run_source(P, a);
        } else if (kGemm && (kind == kGemmBf16 || kind == kGemmSplit)) {
            claim_gemm(P, a);
        } else if (kind == kMandel) {
            claim_mandel(P, a);
        } else if (kind == kFork) {
            run_fork(P, a);
        }
        if (exit_requested(ctl)) return kNone;
    }
    return kNone;
}

// The live-ingress warp: move host messages into mailboxes until the drain
// is quiescent, nothing is published and it has idled long enough (or the
// host asked it to stop).
__device__ void agent_loop(const DrainParams &P) {
    DevCtl *ctl = P.ctl;
    const uint32_t lane = lane_id();
    bool idle = false;
    uint64_t idle_start = 0;
    while (!exit_requested(ctl)) {
        if (poll_host_ring(P)) {
            idle = false;
            continue;
        }
        const uint64_t now = globaltimer();
        if (!idle) {
            idle = true;
            idle_start = now;
        }
        if (quiescent(P)) {
            const bool stop = ld_acquire_sys(&P.hctl->stop) != 0;
            const uint64_t head = ctl->ring_head;
            const bool more = ld_acquire_sys(&P.ring[head & P.ring_mask].seq) == head + 1;
            if (!more && (stop || now - idle_start > P.idle_exit_ns)) {
                if (lane == 0) atomicExch(reinterpret_cast<unsigned int *>(&ctl->exit_flag), 1u);
                break;
            }
        }
        __nanosleep(128);
    }
}

// The persistent drain.  Each CTA has kConsumerWarps consumer warps and one
// producer warp.  In a loop, the consumer warps form a group (team leaders
// claim actors; ring tokens are run on the way), then the producer streams
// the prime table through the CTA's shared-memory ring while every team
// sweeps its batch against it, so one pass over the table serves up to
// kConsumerWarps * K messages.  With the live host ring, warp 0 of CTA 0 is
// the ingress warp and takes no part in groups.
// kSplit: the instantiation for a runtime that splits large factor batches
// (its own kernel, so the sequential sweep's code is the same without it).
template <bool kGemm, bool kSplit>
__global__ void __launch_bounds__(kThreads, kGemm ? 1 : 2) k_drain(DrainParams P) {
    extern __shared__ __align__(128) uint8_t drain_smem[];
    uint8_t *base = drain_smem + ((1024u - (smem_u32(drain_smem) & 1023u)) & 1023u);
    GroupShared &G = *reinterpret_cast<GroupShared *>(base);
    TableTile *ring = reinterpret_cast<TableTile *>(base + kDrainHeader);
    PackedSlots &gslots = *reinterpret_cast<PackedSlots *>(base + kDrainHeader);
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    const bool live0 = P.live && blockIdx.x == 0;
    const bool producer = warp == kConsumerWarps;
    const bool agent = live0 && warp == 0;
    const uint32_t n_cons = live0 ? kConsumerWarps - 1 : kConsumerWarps;
    const uint32_t ci = live0 ? warp - 1 : warp;             // consumer index (consumers only)
    const uint32_t bar_threads = (n_cons + 1) * 32;
    const uint32_t wpb = P.factor_w;
    DevCtl *ctl = P.ctl;
    if (agent) {
        agent_loop(P);
        return;
    }
    if (producer && lane == 0) {
        for (uint32_t i = 0; i < kStages; ++i) {
            mbar_init(&G.full[i], 1);
            mbar_init(&G.empty[i], n_cons);
        }
        fence_barrier_init();
        G.mnext = 0;
        for (uint32_t i = 0; i < kMaxItemsPerRound; ++i) G.msum[i] = 0;
    }
    if constexpr (kGemm) {
        if (producer) gemm_bars_init(G.gb, kPackTmemCols);   // GEMM barriers + tensor memory (warp-wide)
        tc_fence_before();
    }
    const uint32_t gw = blockIdx.x * kConsumerWarps + ci;
    if (!producer && P.batch_count && gw < P.n_routers) {
        route_batch(P, gw);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            add_u32(&ctl->routers_done, 1);
        }
    }
    named_bar_sync(1, bar_threads);
    if constexpr (kGemm) tc_fence_after();
    // teams: consumer warps [j*wpb, (j+1)*wpb); an incomplete last team idles
    const uint32_t team = producer ? 0 : ci / wpb;
    const uint32_t rank = producer ? 0 : ci % wpb;
    const bool team_ok = !producer && (team + 1) * wpb <= n_cons;
    uint32_t t = 0;
    bool idle = false;
    uint64_t idle_start = 0;
    uint32_t idle_ns = 256;
    uint32_t held = kNone;                 // a team leader's claimed batch, kept across GEMM tiles
    uint32_t rng = (blockIdx.x * kWarpsPerCta + warp) * 2654435761u + 1u;   // steal victims
    GemmCounters gk{0, 0, 0, 0};
    uint64_t seen_completed = 0, seen_at = 0;   // completion watchdog (producer lane)
    uint32_t rounds = 0;
    // work items (GEMM packs and tiles, Mandelbrot bands): the GEMM layout runs
    // all three; without it (no GEMM actor) only Mandelbrot bands exist
    const bool item_cta = (kGemm || P.mandel) && !live0;
    for (;;) {
        // ---- form a group: team leaders claim actors (skipped while the GEMM
        // tile queue already holds plenty of work for every CTA)
        if (!producer && team_ok && rank == 0 && held == kNone) {
            bool skip = false;
            if ((kGemm || P.mandel) && lane == 0)
                skip = q_len(&ctl->workq) + q_len(&ctl->packq) > 2 * (int64_t)gridDim.x;
            if (!__shfl_sync(FULL, skip, 0)) held = find_batch<kGemm, kSplit>(P, rng);
        }
        if (!producer && lane == 0) G.batch[ci] = (team_ok && rank == 0) ? held : kNone;
        if (producer) {
            uint32_t ex = 0;
            if (lane == 0) ex = exit_requested(ctl) ? 1u : 0u;
            ex = __shfl_sync(FULL, ex, 0);
            // up to P.gemm_items GEMM items, popped in parallel by as many
            // lanes (one pop's latency); tiles first, so a job's tiles run
            // while its packed operands are still in L2
            uint32_t item = kNone;
            // with fewer items queued than CTAs, each CTA tries one pop, so
            // hundreds of producers do not all reserve (and undo) the last items
            uint32_t npop = 0;
            if (item_cta && !ex) {
                int64_t av = 0;
                if (lane == 0) av = q_len(&ctl->workq) + (kGemm ? q_len(&ctl->packq) : 0);
                av = __shfl_sync(FULL, av, 0);
                if (kGemm) {
                    // GEMM tile runs want full rounds while the queue is not short
                    npop = av >= (int64_t)gridDim.x ? P.gemm_items : (av > 0 ? 1u : 0u);
                } else {
                    // Mandelbrot bands only: an even share, so the last bands of
                    // a step spread over every CTA
                    const int64_t share = av / (int64_t)gridDim.x;
                    npop = share >= (int64_t)P.gemm_items ? P.gemm_items
                                                          : (share > 0 ? (uint32_t)share : (av > 0 ? 1u : 0u));
                }
            }
            if (lane < npop) {
                int pr = q_try_pop(&ctl->workq, P.workq, &item, P.wait_limit_ns);
                if (kGemm && pr == 0) pr = q_try_pop(&ctl->packq, P.packq, &item, P.wait_limit_ns);
                if (pr < 0) fail(P, kErrWaitQueue, 24);
                if (pr <= 0) item = kNone;
            }
            if (P.validation && item != kNone && !work_item_ok(P, item)) {
                bounds_fail(P, 45, item, 0);
                item = kNone;
            }
            // a tile item's job fields, read once here, right after the pop
            // that ordered them, and checked (in every mode: a tile outside
            // its matrix or scratch is refused, not computed)
            TileSnap sn;
            const bool is_tile = kGemm && item != kNone && !(item & (kPackItemFlag | kMandelItemFlag));
            if (is_tile && !tile_snap(P, item, sn)) {
                bounds_fail(P, 47, item, sn.tiles);
                item = kNone;
            }
            const uint32_t got = __ballot_sync(FULL, item != kNone);
            if (item != kNone) {
                const uint32_t pos = __popc(got & ((1u << lane) - 1u));
                G.items[pos] = item;
                if (is_tile) G.snap[pos] = sn;
            }
            if (lane == 0) {
                G.exit = ex;
                G.nitems = __popc(got);
                // watchdog: busy warps can keep the heartbeat fresh without any
                // message completing; give up if nothing completes for a long
                // time (checked when idle, and every 64th round)
                if (got == 0 || (++rounds & 63u) == 0) {
                    const uint64_t done_now = ld_relaxed_gpu(&ctl->completed);
                    const uint64_t tnow = globaltimer();
                    if (done_now != seen_completed || seen_at == 0 || quiescent(P)) {
                        seen_completed = done_now;
                        seen_at = tnow;
                    } else if (tnow > seen_at && tnow - seen_at > kCompletionLimitNs) {
                        fail(P, kErrNoCompletion, 20, done_now, ld_acquire_gpu(&ctl->ingested));
                    }
                }
            }
        }
        named_bar_sync(1, bar_threads);
        if (G.exit) break;
        if (const uint32_t ni = G.nitems) {
            // items first: short, and other CTAs may wait on the same job
            if constexpr (!kGemm) {
                // only Mandelbrot bands exist without the GEMM layout
                drain_mandel_bands(P, G, &G.items[0], ni, bar_threads);
            } else {
                for (uint32_t i = 0; i < ni;) {
                    const uint32_t it = G.items[i];
                    if (it & kPackItemFlag) {
                        drain_gemm_pack(P, gslots, it, bar_threads);
                        ++i;
                    } else if (it & kMandelItemFlag) {
                        // Mandelbrot bands: the round's bands are one pool
                        // (the queue order puts a job's bands together)
                        uint32_t e = i + 1;
                        while (e < ni && (G.items[e] & kMandelItemFlag) && !(G.items[e] & kPackItemFlag)) ++e;
                        drain_mandel_bands(P, G, &G.items[i], e - i, bar_threads);
                        i = e;
                    } else {
                        // consecutive tiles run as one pipeline
                        uint32_t e = i + 1;
                        while (e < ni && !(G.items[e] & (kPackItemFlag | kMandelItemFlag))) ++e;
                        drain_gemm_tiles(P, G, gslots, &G.items[i], &G.snap[i], e - i, gk, bar_threads);
                        i = e;
                    }
                }
            }
            idle = false;
            idle_ns = 256;
            continue;
        }
        uint32_t mine = kNone;
        if (!producer) mine = team_ok ? G.batch[team * wpb] : kNone;
        if (producer && lane == 0) {
            uint32_t active = 0, limit = 0;
            for (uint32_t i = 0; i < n_cons; ++i) {
                const uint32_t tb = i / wpb;
                if ((tb + 1) * wpb > n_cons) continue;
                const uint32_t enc = G.batch[tb * wpb];
                if (enc == kNone) continue;
                ++active;
                limit = max(limit, P.batches[enc & 0xFFFFFFu].maxbound);
            }
            G.active = active;
            G.limit_tiles = (limit + kTile - 1) / kTile;
            G.final_tile = 0xFFFFFFFFu;
        }
        named_bar_sync(1, bar_threads);
        if (G.active == 0) {
            // nothing to sweep in this CTA: exit when the drain is quiescent
            if (producer && lane == 0) {
                const uint64_t now = globaltimer();
                if (!idle) {
                    idle = true;
                    idle_start = now;
                }
                if (quiescent(P)) {
                    if (!P.live) atomicExch(reinterpret_cast<unsigned int *>(&ctl->exit_flag), 1u);
                } else {
                    const uint64_t hb = *((volatile uint64_t *)&ctl->heartbeat);
                    const uint64_t last = hb > idle_start ? hb : idle_start;
                    // another warp's heartbeat may be newer than `now`
                    if (last < now && now - last > P.wait_limit_ns)
                        fail(P, kErrStall, 8, ld_acquire_gpu(&ctl->ingested), ld_acquire_gpu(&ctl->completed));
                }
            }
            // back off: idle CTAs would otherwise take issue slots from
            // sweeping CTAs on the same SM
            __nanosleep(idle_ns);
            idle_ns = min(idle_ns * 2, 2000u);
            continue;
        }
        idle = false;
        idle_ns = 256;
        // ---- sweep
        if (producer) {
            uint32_t tt = t;
            if (lane == 0) {
                if constexpr (kSplit) group_produce_split(P, G, ring, tt, n_cons, wpb);
                else group_produce(P, G, ring, tt);
            }
            t = __shfl_sync(FULL, tt, 0);
        } else {
            group_consume<kSplit>(P, G, ring, t, mine, rank, wpb);
        }
        held = kNone;
        named_bar_sync(1, bar_threads);
    }
    if constexpr (kGemm) {
        // release tensor memory (after every tcgen05 operation of this CTA)
        tc_fence_before();
        named_bar_sync(1, bar_threads);
        if (producer) {
            tc_fence_after();
            tmem_dealloc(G.gb.tmem, kPackTmemCols);
        }
    }
}

// ---------------------------------------------------------------------------
// Per-message launch (the comparator): one kernel launch factors one n with
// the whole grid.  Warp g tests chunks g, g + G, ... of 32 primes and
// records the smallest dividing index with atomicMin in scratch[0]; the last
// CTA to finish writes the reply and resets the scratch words for the next
// launch.  scratch = {found, ctas_done} (two uint32 words, zero/kNoFactor at
// rest).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kOneThreads) k_factor_one(uint64_t n, const uint32_t *primes,
                                                          const uint32_t *pinv, const uint32_t *plim,
                                                          uint32_t nprimes, uint64_t reply_addr,
                                                          uint32_t reply_token, uint64_t tag,
                                                          uint32_t *scratch, DevCtl *ctl) {
    const uint32_t lane = lane_id();
    const bool even = (n >= 4) && !(n & 1u);
    const uint32_t bound = even ? 0 : factor_bound(primes, nprimes, n);
    const uint32_t gw = blockIdx.x * (kOneThreads / 32) + (threadIdx.x >> 5);
    const uint32_t nw = gridDim.x * (kOneThreads / 32);
    const uint32_t nl = 0u - (uint32_t)n;
    uint64_t tests = 0;
    for (uint32_t c = gw * 32; c < bound; c += nw * 32) {
        if (*((volatile uint32_t *)&scratch[0]) < c) break;
        const uint32_t idx = c + lane;
        const bool hit = idx < bound && mont_divides(n, nl, __ldg(primes + idx), __ldg(pinv + idx), __ldg(plim + idx));
        tests += 32;
        const uint32_t mn = __reduce_min_sync(FULL, hit ? idx : 0xFFFFFFFFu);
        if (mn != 0xFFFFFFFFu) {
            if (lane == 0) atomicMin(reinterpret_cast<unsigned int *>(&scratch[0]), mn);
            break;
        }
    }
    if (lane == 0 && tests) add_u64(&ctl->prime_tests, tests);
    __syncthreads();
    __shared__ uint32_t last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(reinterpret_cast<unsigned int *>(&scratch[1]), 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const uint32_t found = *((volatile uint32_t *)&scratch[0]);
        int32_t st;
        uint64_t r0, r1;
        factor_result(n, even, found, bound, primes, &st, &r0, &r1);
        write_reply(reply_addr, st, r0, r1, tag, reply_token);
        scratch[0] = kNoFactor;
        scratch[1] = 0;
        add_u64(&ctl->messages, 1);
        __threadfence();
    }
}

// Per-message launch of one ring-token message: the same handler as the
// drain, run by one warp; its outgoing messages go to `outbox` (pinned host
// memory) for the host to launch next.  outbox[0].seq counts entries.
__global__ void k_token_one(ActorDesc *actors, uint32_t a, uint32_t kind, int32_t v,
                            uint64_t reply_addr, uint32_t reply_token, IngressEntry *outbox,
                            DevCtl *ctl) {
    if (threadIdx.x != 0) return;
    ActorDesc *A = &actors[a];
    uint32_t nout = 0;
    auto emit = [&](uint32_t to, uint32_t k, uint64_t payload, uint64_t raddr, uint32_t tok, uint64_t tag) {
        IngressEntry *e = &outbox[1 + nout++];
        e->actor = to;
        e->kind = k;
        e->payload = payload;
        e->reply_addr = raddr;
        e->reply_token = tok;
        e->tag = tag;
        e->sender = 0x80000000u | a;
    };
    auto emit_factor = [&]() {
        if (!(A->flags & kActorMaster)) return;
        const uint32_t k = A->round;
        if (k >= A->factor_count) return;
        A->round = k + 1;
        emit(A->worker, kFactor, reinterpret_cast<const uint64_t *>(A->factor_n)[k],
             A->factor_replies + (uint64_t)k * sizeof(Reply), 1, k);
    };
    if (A->state == kDone) {
        write_reply(reply_addr, 2, 0, 0, 0, reply_token);
    } else {
        if ((kind >> 16) & kMsgStart) {
            emit_factor();
            emit(A->next, kToken, (uint32_t)v, 0, 0, 0);
        } else if (v > 0) {
            emit_factor();
            emit(A->next, kToken, (uint32_t)(v - 1), 0, 0, 0);
        } else {
            A->state = kDone;
            if (actors[A->next].state != kDone) emit(A->next, kToken, 0, 0, 0, 0);
        }
        A->user_state = v;
        write_reply(reply_addr, 0, (uint32_t)v, 0, 0, reply_token);
    }
    add_u64(&ctl->messages, 1);
    __threadfence_system();
    st_release_sys(&outbox[0].seq, nout);
}

// Reset ring actors to their spawn state (stream-ordered; graph-capturable).
__global__ void k_reset_actors(ActorDesc *actors, uint32_t n_actors) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_actors) return;
    ActorDesc *A = &actors[i];
    if (A->kind == kToken) {
        A->state = kWaiting;
        A->user_state = A->init_state;
        A->round = 0;
        A->head = A->tail;
        A->ring_inc = 0;
        A->ring_live = 0;
    } else if (A->kind == kSink) {
        A->sink_count = 0;
        A->sink_sum = 0;
    } else if (A->kind == kFork) {
        A->user_state = 0;
        A->sink_count = 0;
        A->sink_sum = 0;
    }
}

// Set up the FORK actor pool: ids base .. base + count - 1, free (DONE), each
// with kForkSlots mailbox slots starting at slot0 + kForkSlots * i.
__global__ void k_fork_pool_init(ActorDesc *actors, uint32_t base, uint32_t count, uint64_t slot0) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        ActorDesc d{};
        d.kind = kFork;
        d.state = kDone;
        d.cap_mask = kForkSlots - 1;
        d.slot_base = slot0 + (uint64_t)kForkSlots * i;
        d.next = kNone;
        actors[base + i] = d;
    }
}

// Record the device clock in stream order.
__global__ void k_mark(DevCtl *ctl) { ctl->t_mark = globaltimer(); }

// Reset the counters a drain launch reads (stream-ordered).
__global__ void k_reset_ctl(DevCtl *ctl) {
    ctl->exit_flag = 0;
    ctl->routers_done = 0;
    ctl->heartbeat = 0;
}

// ---------------------------------------------------------------------------
// Prime table: segmented sieve of Eratosthenes over the odd numbers.  Bit i
// of the global bitmap stands for 2i + 1 and is set when composite (or 1).
// ---------------------------------------------------------------------------
constexpr uint32_t kSegBits = 1u << 18;

__global__ void k_sieve(uint32_t *bits, uint64_t nbits, const uint32_t *small, uint32_t nsmall) {
    extern __shared__ uint32_t seg[];
    const uint64_t i0 = (uint64_t)blockIdx.x * kSegBits;
    const uint32_t words = kSegBits / 32;
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) seg[w] = 0;
    __syncthreads();
    const uint64_t lo = 2 * i0 + 1;                     // first odd number of the segment
    const uint64_t hi = 2 * (i0 + kSegBits) - 1;        // last odd number
    for (uint32_t k = threadIdx.x; k < nsmall; k += blockDim.x) {
        const uint64_t p = small[k];
        if (p * p > hi) break;
        uint64_t m = (lo + p - 1) / p * p;
        if (!(m & 1)) m += p;
        if (m < p * p) m = p * p;
        for (uint64_t x = m; x <= hi; x += 2 * p) {
            const uint32_t b = (uint32_t)((x - lo) >> 1);
            atomicOr(&seg[b >> 5], 1u << (b & 31));
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) seg[0] |= 1u;  // 1 is not prime
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
        const uint64_t gbit = i0 + (uint64_t)w * 32;
        if (gbit < nbits) {
            uint32_t v = seg[w];
            if (gbit + 32 > nbits) v |= ~0u << (uint32_t)(nbits - gbit);  // beyond the limit
            bits[gbit >> 5] = v;
        }
    }
}

// Primes per segment (count of zero bits).
__global__ void k_sieve_count(const uint32_t *bits, uint64_t nwords, uint32_t *counts) {
    __shared__ uint32_t tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    const uint64_t w0 = (uint64_t)blockIdx.x * (kSegBits / 32);
    uint32_t c = 0;
    for (uint32_t w = threadIdx.x; w < kSegBits / 32; w += blockDim.x)
        if (w0 + w < nwords) c += __popc(~bits[w0 + w]);
    atomicAdd(&tot, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

// Write the primes of each segment at its offset, with p^-1 mod 2^32 (Newton
// iteration x <- x(2 - p x), 3 -> 6 -> 12 -> 24 -> 48 correct bits) and
// floor((2^32 - 1) / p).
__global__ void k_sieve_emit(const uint32_t *bits, uint64_t nwords, const uint32_t *offsets,
                             uint32_t *primes, uint32_t *pinv, uint32_t *plim) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t running;
    const uint64_t w0 = (uint64_t)blockIdx.x * (kSegBits / 32);
    if (threadIdx.x == 0) running = offsets[blockIdx.x];
    __syncthreads();
    for (uint32_t base = 0; base < kSegBits / 32; base += blockDim.x) {
        const uint64_t w = w0 + base + threadIdx.x;
        uint32_t v = (base + threadIdx.x < kSegBits / 32 && w < nwords) ? ~bits[w] : 0u;
        const uint32_t c = __popc(v);
        // block exclusive scan of c
        uint32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if ((threadIdx.x & 31) >= (uint32_t)o) incl += t;
        }
        if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t nwarps = blockDim.x >> 5;
            uint32_t x = threadIdx.x < nwarps ? warp_tot[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, x, o);
                if (threadIdx.x >= (uint32_t)o) x += t;
            }
            warp_tot[threadIdx.x] = x;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t warp_excl = (threadIdx.x >= 32) ? warp_tot[(threadIdx.x >> 5) - 1] : 0;
        uint32_t pos = running + warp_excl + incl - c;
        while (v) {
            const uint32_t b = __ffs(v) - 1;
            v &= v - 1;
            const uint32_t p = (uint32_t)(2 * (w * 32 + b) + 1);
            uint32_t x = p;  // p*p == 1 mod 8 for odd p: 3 correct bits
            x *= 2u - p * x;
            x *= 2u - p * x;
            x *= 2u - p * x;
            x *= 2u - p * x;
            primes[pos] = p;
            pinv[pos] = x;
            plim[pos] = 0xFFFFFFFFu / p;
            ++pos;
        }
        __syncthreads();
        if (threadIdx.x == 0) running += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
}

// A kernel that waits, bounded, for a flag that nothing sets, and reports
// the expiry through the error word (exercises the bounded-wait path).
__global__ void k_debug_wait(const uint32_t *flag, uint64_t limit_ns, DevCtl *ctl, HostCtl *hctl) {
    if (threadIdx.x != 0) return;
    WaitClock w(limit_ns);
    while (ld_acquire_gpu(flag) == 0) {
        if (!w.again()) {
            raise_error(ctl, kErrDebugWait, 9);
            st_release_sys(&hctl->error_word, *((volatile uint32_t *)&ctl->error_word));
            return;
        }
    }
}

}  // namespace cafgpu

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
#include <vector>

#include "kernels.h"

namespace cafgpu {

static cudaError_t drain_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_drain<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kDrainSmemFactor);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_drain<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDrainSmemMixed);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_drain<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDrainSmemFactor);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_drain<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDrainSmemMixed);
    if (e == cudaSuccess) done = true;
    return e;
}

// Resident CTAs per SM of the instantiation launch_drain runs for (gemm, split).
cudaError_t drain_occupancy(bool gemm, bool split, int *ctas_per_sm) {
    cudaError_t e = drain_attr();
    if (e != cudaSuccess) return e;
    if (gemm && split)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_drain<true, true>, kThreads,
                                                             kDrainSmemMixed);
    if (gemm)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_drain<true, false>, kThreads,
                                                             kDrainSmemMixed);
    if (split)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_drain<false, true>, kThreads,
                                                             kDrainSmemFactor);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_drain<false, false>, kThreads,
                                                         kDrainSmemFactor);
}

cudaError_t launch_drain(const DrainParams &p, unsigned grid, cudaStream_t stream) {
    cudaError_t e = drain_attr();
    if (e != cudaSuccess) return e;
    const bool split = p.split > 1;
    if (p.gemm && split)
        k_drain<true, true><<<grid, kThreads, kDrainSmemMixed, stream>>>(p);
    else if (p.gemm)
        k_drain<true, false><<<grid, kThreads, kDrainSmemMixed, stream>>>(p);
    else if (split)
        k_drain<false, true><<<grid, kThreads, kDrainSmemFactor, stream>>>(p);
    else
        k_drain<false, false><<<grid, kThreads, kDrainSmemFactor, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fork_pool_init(ActorDesc *actors, uint32_t base, uint32_t count, uint64_t slot0,
                                  cudaStream_t stream) {
    k_fork_pool_init<<<1024, 256, 0, stream>>>(actors, base, count, slot0);
    return cudaGetLastError();
}

cudaError_t launch_mark(DevCtl *ctl, cudaStream_t stream) {
    k_mark<<<1, 1, 0, stream>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_reset_ctl(DevCtl *ctl, cudaStream_t stream) {
    k_reset_ctl<<<1, 1, 0, stream>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_factor_one(uint64_t n, const uint32_t *primes, const uint32_t *pinv,
                              const uint32_t *plim, uint32_t nprimes, uint64_t reply_addr,
                              uint32_t reply_token, uint64_t tag, uint32_t *scratch, DevCtl *ctl,
                              unsigned grid, cudaStream_t stream) {
    k_factor_one<<<grid, kOneThreads, 0, stream>>>(n, primes, pinv, plim, nprimes, reply_addr, reply_token,
                                                tag, scratch, ctl);
    return cudaGetLastError();
}

cudaError_t launch_token_one(ActorDesc *actors, uint32_t a, uint32_t kind, int32_t v,
                             uint64_t reply_addr, uint32_t reply_token, IngressEntry *outbox,
                             DevCtl *ctl, cudaStream_t stream) {
    k_token_one<<<1, 32, 0, stream>>>(actors, a, kind, v, reply_addr, reply_token, outbox, ctl);
    return cudaGetLastError();
}

cudaError_t launch_reset_actors(ActorDesc *actors, uint32_t n_actors, cudaStream_t stream) {
    if (n_actors == 0) return cudaSuccess;
    k_reset_actors<<<(n_actors + 255) / 256, 256, 0, stream>>>(actors, n_actors);
    return cudaGetLastError();
}

cudaError_t launch_debug_wait(const uint32_t *flag, uint64_t limit_ns, DevCtl *ctl, HostCtl *hctl,
                              cudaStream_t stream) {
    k_debug_wait<<<1, 32, 0, stream>>>(flag, limit_ns, ctl, hctl);
    return cudaGetLastError();
}

cudaError_t build_prime_table(uint64_t limit, uint32_t pad, uint32_t **primes, uint32_t **pinv,
                              uint32_t **plim, uint32_t *count, cudaStream_t stream) {
    *primes = *pinv = *plim = nullptr;
    *count = 0;
    if (limit < 3) limit = 3;
    // small odd primes up to sqrt(limit), host sieve
    uint64_t r = 1;
    while ((r + 1) * (r + 1) <= limit) ++r;
    std::vector<uint8_t> comp(r + 1, 0);
    std::vector<uint32_t> small;
    for (uint64_t i = 2; i <= r; ++i) {
        if (comp[i]) continue;
        if (i > 2) small.push_back((uint32_t)i);
        for (uint64_t j = i * i; j <= r; j += i) comp[j] = 1;
    }
    const uint64_t nbits = (limit + 1) / 2;  // odd numbers 1, 3, ..., <= limit
    const uint64_t nwords = (nbits + 31) / 32;
    const uint32_t nseg = (uint32_t)((nbits + kSegBits - 1) / kSegBits);
    uint32_t *d_small = nullptr, *d_bits = nullptr, *d_counts = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_small, sizeof(uint32_t) * (small.size() + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_bits, sizeof(uint32_t) * nwords)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d_counts, sizeof(uint32_t) * nseg)) != cudaSuccess) return e;
    if (!small.empty())
        cudaMemcpyAsync(d_small, small.data(), sizeof(uint32_t) * small.size(), cudaMemcpyHostToDevice, stream);
    cudaFuncSetAttribute(k_sieve, cudaFuncAttributeMaxDynamicSharedMemorySize, kSegBits / 8);
    k_sieve<<<nseg, 512, kSegBits / 8, stream>>>(d_bits, nbits, d_small, (uint32_t)small.size());
    k_sieve_count<<<nseg, 256, 0, stream>>>(d_bits, nwords, d_counts);
    std::vector<uint32_t> counts(nseg), offsets(nseg);
    cudaMemcpyAsync(counts.data(), d_counts, sizeof(uint32_t) * nseg, cudaMemcpyDeviceToHost, stream);
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
    uint64_t total = 0;
    for (uint32_t s = 0; s < nseg; ++s) {
        offsets[s] = (uint32_t)total;
        total += counts[s];
    }
    const size_t bytes = sizeof(uint32_t) * (total + pad);
    if ((e = cudaMalloc(primes, bytes)) != cudaSuccess) return e;
    if ((e = cudaMalloc(pinv, bytes)) != cudaSuccess) return e;
    if ((e = cudaMalloc(plim, bytes)) != cudaSuccess) return e;
    cudaMemsetAsync(*primes, 0, bytes, stream);
    cudaMemsetAsync(*pinv, 0, bytes, stream);
    cudaMemsetAsync(*plim, 0, bytes, stream);
    cudaMemcpyAsync(d_counts, offsets.data(), sizeof(uint32_t) * nseg, cudaMemcpyHostToDevice, stream);
    k_sieve_emit<<<nseg, 256, 0, stream>>>(d_bits, nwords, d_counts, *primes, *pinv, *plim);
    e = cudaStreamSynchronize(stream);
    cudaFree(d_small);
    cudaFree(d_bits);
    cudaFree(d_counts);
    *count = (uint32_t)total;
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace cafgpu
