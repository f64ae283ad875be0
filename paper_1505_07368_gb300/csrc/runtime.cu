// Host runtime behind caf_gpu.h: device arenas, actor table, host ingress
// ring, reply slots, the two backends (persistent drain and one launch per
// message) and the C entry points.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/caf_gpu.h"
#include "isqrt.h"
#include "kernels.h"
#include "layout.h"
#include "mandel.cuh"

using namespace cafgpu;

namespace {

uint32_t next_pow2(uint64_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }

constexpr uint32_t kMaxGemmN = 1u << 15;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

template <class T>
T load_acquire(const T *p) {
    return __atomic_load_n(p, __ATOMIC_ACQUIRE);
}

}  // namespace

struct caf_gpu_runtime {
    caf_gpu_runtime_cfg cfg{};
    // guard regions after the device arrays: (allocation base, guard start)
    std::vector<std::pair<void *, uint8_t *>> guards;
    int device = 0;
    int n_sms = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t setup = nullptr;
    bool own_stream = false;
    unsigned grid = 0;

    // device arena
    DevCtl *d_ctl = nullptr;
    ActorDesc *d_actors = nullptr;
    Slot *d_slots = nullptr;
    uint64_t n_slots = 0, slots_used = 0;
    QCell *d_readyq = nullptr, *d_freeq = nullptr, *d_workq = nullptr, *d_packq = nullptr;
    uint32_t readyq_cap = 0, freeq_cap = 0, workq_cap = 0;
    FactorBatch *d_batches = nullptr;
    uint32_t n_batches = 0;
    GemmJob *d_jobs = nullptr;
    MandelJob *d_mjobs = nullptr;
    QCell *d_mjobq = nullptr;
    QCell *d_forkq = nullptr;              // free ids of the FORK actor pool
    QCell *d_segq = nullptr;               // segments of split factor batches
    uint32_t fork_base = 0, fork_pool = 0; // pool ids fork_base .. fork_base + fork_pool - 1 (0: no pool yet)
    bool graphs_made = false;              // a CUDA graph holds the current table addresses
    QueueHdr *d_localq_hdr = nullptr;      // work stealing: a ready queue per CTA
    QCell *d_localq = nullptr;
    QCell *d_jobq = nullptr, *d_jobq_large = nullptr;
    uint32_t jobq_cap = 0;
    uint8_t *d_pack_small = nullptr, *d_pack_large = nullptr;   // packed-operand scratch of the job records
    bool gemm_enabled = false;             // a GEMM actor exists: drains use the GEMM layout
    bool mandel_enabled = false;           // a MANDELBROT actor exists: drains run work items
    uint32_t n_factor_actors = 0;          // FACTOR actors spawned (teams of factor_warps need them)
    unsigned grid_factor = 0, grid_mixed = 0;
    uint32_t *d_primes = nullptr, *d_pinv = nullptr, *d_plim = nullptr;
    uint32_t nprimes = 0;
    uint64_t prime_limit = 0;
    LogRow *d_log = nullptr;
    uint32_t *d_scratch = nullptr;
    uint32_t *d_zero = nullptr;

    // host mirror of the actor table
    std::vector<ActorDesc> actors;
    uint32_t n_actors = 0;

    // pinned, device-visible
    IngressEntry *ring = nullptr;
    HostCtl *hctl = nullptr;
    Reply *replies = nullptr;
    GemmDesc *gemm_descs = nullptr;        // one per reply slot (host GEMM requests)
    MandelDesc *mandel_descs = nullptr;    // one per reply slot (host Mandelbrot requests)
    IngressEntry *outbox = nullptr;
    uint32_t outbox_per_msg = 4;
    uint32_t outbox_msgs = 256;

    std::mutex mu;                 // ring tickets, sender counters, reply slots, launches
    uint64_t ring_tail = 0;
    std::unordered_map<uint32_t, uint32_t> sender_seq;
    std::vector<uint32_t> free_slots;
    std::vector<uint32_t> gen;
    std::vector<uint8_t> in_use;

    int backend = CAF_GPU_BACKEND_PERSISTENT;
    cudaEvent_t live_done = nullptr;
    bool live_launched = false;
    uint64_t launches = 0;
    DevCtl last_stats{};

    // per-message backend: messages produced by token kernels, waiting for a launch
    std::deque<IngressEntry> pm_pending;

    bool capturing = false;                // between caf_gpu_graph_begin and _end
};

struct caf_gpu_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return CAF_GPU_ECUDA; \
    } while (0)

DrainParams make_params(caf_gpu_runtime *rt) {
    DrainParams p{};
    p.ctl = rt->d_ctl;
    p.actors = rt->d_actors;
    p.n_actors = rt->n_actors;
    p.slots = rt->d_slots;
    p.readyq = rt->d_readyq;
    p.freeq = rt->d_freeq;
    p.workq = rt->d_workq;
    p.packq = rt->d_packq;
    p.batches = rt->d_batches;
    p.primes = rt->d_primes;
    p.pinv = rt->d_pinv;
    p.plim = rt->d_plim;
    p.nprimes = rt->nprimes;
    p.factor_k = rt->cfg.factor_batch;
    // warps share factor batches in teams; without factor actors every
    // consumer warp leads its own team, so every warp claims actors
    p.factor_w = rt->n_factor_actors ? rt->cfg.factor_warps : 1u;
    p.max_claim = rt->cfg.max_msgs_per_claim;
    p.gemm_items = rt->cfg.gemm_items_per_round;
    p.gemm_wide = rt->cfg.gemm_tile_n == 256 ? 1u : 0u;
    p.max_n = rt->cfg.max_factor_n;
    p.wait_limit_ns = rt->cfg.wait_limit_ns;
    p.idle_exit_ns = rt->cfg.idle_exit_ns;
    p.log = rt->d_log;
    p.log_capacity = rt->d_log ? rt->cfg.log_capacity : 0;
    p.validation = rt->cfg.validation_mode ? 1 : 0;
    p.ring = rt->ring;
    p.hctl = rt->hctl;
    p.ring_mask = rt->cfg.ingress_capacity - 1;
    p.jobs = rt->d_jobs;
    p.jobq = rt->d_jobq;
    p.jobq_large = rt->d_jobq_large;
    p.mjobs = rt->d_mjobs;
    p.mjobq = rt->d_mjobq;
    p.forkq = rt->d_forkq;
    p.segq = rt->d_segq;
    // factor_split 0 (automatic): no split unless a launch chooses it
    p.split = rt->cfg.factor_split == 0 ? 1u : rt->cfg.factor_split;
    p.n_slots = rt->n_slots + (uint64_t)kForkSlots * rt->fork_pool;
    p.n_batches = rt->n_batches;
    p.localq_hdr = rt->d_localq_hdr;
    p.localq = rt->d_localq;
    p.localq_cap = kLocalQueueCap;
    p.steal = rt->d_localq ? 1u : 0u;
    p.fork_base = rt->fork_base;
    p.fork_pool = rt->fork_pool;
    p.pack_small = rt->d_pack_small;
    p.pack_large = rt->d_pack_large;
    p.gemm = rt->gemm_enabled ? 1u : 0u;
    p.mandel = rt->mandel_enabled ? 1u : 0u;
    return p;
}

unsigned drain_grid(caf_gpu_runtime *rt) { return rt->gemm_enabled ? rt->grid_mixed : rt->grid_factor; }

// Host status for a nonzero device error word: a refused out-of-range index
// (validation mode) or an expired bounded wait.
int device_error(uint32_t word) { return (word & 0xFFu) == kErrBounds ? CAF_GPU_EBOUNDS : CAF_GPU_EWAITLIMIT; }

// Device arrays are allocated with a guard region of kGuardBytes after them,
// filled with kGuardByte.  No kernel writes there; check_guards reads every
// guard back, so a write past the end of an array shows up as a changed
// guard (the runtime's arena canaries).
constexpr uint64_t kGuardBytes = 256;
constexpr uint8_t kGuardByte = 0xA5;

cudaError_t guarded_malloc(caf_gpu_runtime *rt, void **p, uint64_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes + kGuardBytes);
    if (e != cudaSuccess) return e;
    uint8_t *g = static_cast<uint8_t *>(*p) + bytes;
    e = cudaMemset(g, kGuardByte, kGuardBytes);
    if (e != cudaSuccess) {
        cudaFree(*p);
        *p = nullptr;
        return e;
    }
    rt->guards.emplace_back(*p, g);
    return cudaSuccess;
}
template <class T>
cudaError_t guarded_malloc(caf_gpu_runtime *rt, T **p, uint64_t bytes) {
    return guarded_malloc(rt, reinterpret_cast<void **>(p), bytes);
}

// Forget the guard of an allocation about to be freed.
void drop_guard(caf_gpu_runtime *rt, void *base) {
    for (size_t i = 0; i < rt->guards.size(); ++i)
        if (rt->guards[i].first == base) {
            rt->guards.erase(rt->guards.begin() + (long)i);
            return;
        }
}

// Guards whose bytes changed (-1 if they cannot be read).
int check_guards(caf_gpu_runtime *rt) {
    int bad = 0;
    uint8_t h[kGuardBytes];
    for (auto &g : rt->guards) {
        if (cudaMemcpy(h, g.second, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
        for (uint64_t i = 0; i < kGuardBytes; ++i)
            if (h[i] != kGuardByte) {
                ++bad;
                break;
            }
    }
    return bad;
}

int init_queue(caf_gpu_runtime *rt, QCell **cells, uint32_t cap, QueueHdr *hdr_dev,
               const std::vector<uint32_t> &initial) {
    std::vector<QCell> h(cap);
    for (uint32_t i = 0; i < cap; ++i) {
        h[i].seq = i;
        h[i].val = 0;
        h[i].pad = 0;
    }
    for (size_t i = 0; i < initial.size(); ++i) {
        h[i].seq = i + 1;
        h[i].val = initial[i];
    }
    CK(guarded_malloc(rt, cells, sizeof(QCell) * cap));
    CK(cudaMemcpy(*cells, h.data(), sizeof(QCell) * cap, cudaMemcpyHostToDevice));
    QueueHdr q{};
    q.enq = initial.size();
    q.deq = 0;
    q.avail = (int64_t)initial.size();
    q.mask = cap - 1;
    CK(cudaMemcpy(hdr_dev, &q, sizeof(q), cudaMemcpyHostToDevice));
    return 0;
}

int launch_live(caf_gpu_runtime *rt) {
    DrainParams p = make_params(rt);
    p.live = 1;
    CK(launch_reset_ctl(rt->d_ctl, rt->stream));
    CK(launch_drain(p, drain_grid(rt), rt->stream));
    CK(cudaEventRecord(rt->live_done, rt->stream));
    rt->live_launched = true;
    rt->launches += 2;
    return 0;
}

bool live_running(caf_gpu_runtime *rt) {
    return rt->live_launched && cudaEventQuery(rt->live_done) == cudaErrorNotReady;
}

// Launch the persistent drain if host messages are waiting and no drain runs.
// Caller holds rt->mu.
int kick_locked(caf_gpu_runtime *rt) {
    if (rt->backend != CAF_GPU_BACKEND_PERSISTENT) return 0;
    if (live_running(rt)) return 0;
    if (load_acquire(&rt->hctl->ring_consumed) == rt->ring_tail) return 0;
    return launch_live(rt);
}

int kick(caf_gpu_runtime *rt) {
    std::lock_guard<std::mutex> g(rt->mu);
    return kick_locked(rt);
}

int check_msg(caf_gpu_runtime *rt, caf_gpu_actor to, const caf_gpu_msg *m, uint32_t *idx) {
    if (!rt || !m) return CAF_GPU_EINVAL;
    if (to == 0 || to > rt->n_actors) return CAF_GPU_EINVAL;
    const uint32_t a = (uint32_t)(to - 1);
    const ActorDesc &d = rt->actors[a];
    if (m->kind != d.kind) return CAF_GPU_EINVAL;
    if (m->kind == kFactor && m->u64 > rt->cfg.max_factor_n) return CAF_GPU_EINVAL;
    if (m->kind == kGemmBf16 || m->kind == kGemmSplit) {
        if (!m->A || !m->B || !m->C || m->n == 0 || m->n > kMaxGemmN) return CAF_GPU_EINVAL;
        if (rt->backend == CAF_GPU_BACKEND_PERSISTENT && m->n > kMaxDrainGemmN) return CAF_GPU_EINVAL;
    }
    if ((m->kind == kSink || m->kind == kSource) && rt->backend != CAF_GPU_BACKEND_PERSISTENT)
        return CAF_GPU_EINVAL;
    if (m->kind == kFork) {
        // a computation whose tree fits the device actor pool; persistent backend only
        if (rt->backend != CAF_GPU_BACKEND_PERSISTENT) return CAF_GPU_EINVAL;
        if (m->flags || m->u64 > kForkMaxN || (2ull << m->u64) - 2 > rt->fork_pool) return CAF_GPU_EINVAL;
    }
    if (m->kind == kMandel) {
        // the descriptor is read (copied) at the call
        if (!m->u64) return CAF_GPU_EINVAL;
        if (!mandel_desc_ok(*reinterpret_cast<const MandelDesc *>(m->u64))) return CAF_GPU_EINVAL;
    }
    if (m->kind == kSource && m->u64 > 0xFFFFFFFFull) return CAF_GPU_EINVAL;
    if (m->kind == kToken) {
        // token values fit 31 bits; a re-creating master runs in the drain only
        if (m->u64 > 0x7FFFFFFFull) return CAF_GPU_EINVAL;
        if ((d.flags & kActorRecreate) && rt->backend != CAF_GPU_BACKEND_PERSISTENT) return CAF_GPU_EINVAL;
        uint32_t state = 0;
        if (cudaMemcpy(&state, &rt->d_actors[a].state, sizeof(state), cudaMemcpyDeviceToHost) != cudaSuccess)
            return CAF_GPU_ECUDA;
        if (state == kDone) return CAF_GPU_EDEAD;
    }
    *idx = a;
    return 0;
}

uint32_t factor_grid(caf_gpu_runtime *rt, uint64_t n) {
    // about one chunk of 32 primes per warp: primes below sqrt(n) ~ s / ln s
    const double s = std::sqrt((double)n);
    const double np = s > 3 ? s / std::log(s) : 1.0;
    uint64_t g = (uint64_t)(np / 32.0 / (kOneThreads / 32)) + 1;
    return (uint32_t)std::min<uint64_t>(g, (uint64_t)rt->n_sms * 4);
}

// Launch the handler for one message (per-message backend).  Caller holds rt->mu.
int pm_launch(caf_gpu_runtime *rt, const IngressEntry &e, uint32_t outbox_index) {
    const uint32_t kind = e.kind & 0xFFFFu;
    if (kind == kFactor) {
        CK(launch_factor_one(e.payload, rt->d_primes, rt->d_pinv, rt->d_plim, rt->nprimes, e.reply_addr,
                             e.reply_token, e.tag, rt->d_scratch, rt->d_ctl, factor_grid(rt, e.payload),
                             rt->stream));
    } else if (kind == kToken) {
        IngressEntry *ob = rt->outbox + (size_t)outbox_index * rt->outbox_per_msg;
        ob[0].seq = ~0ull;
        CK(launch_token_one(rt->d_actors, e.actor, e.kind, (int32_t)(uint32_t)e.payload, e.reply_addr,
                            e.reply_token, ob, rt->d_ctl, rt->stream));
    } else {
        return CAF_GPU_EINVAL;
    }
    rt->launches += 1;
    return 0;
}

// Per-message backend: run every pending token message in waves until no
// more are produced.  Caller holds rt->mu.
int pm_pump(caf_gpu_runtime *rt) {
    while (!rt->pm_pending.empty()) {
        std::vector<IngressEntry> wave;
        while (!rt->pm_pending.empty() && wave.size() < rt->outbox_msgs) {
            wave.push_back(rt->pm_pending.front());
            rt->pm_pending.pop_front();
        }
        for (uint32_t i = 0; i < wave.size(); ++i) {
            int r = pm_launch(rt, wave[i], i);
            if (r) return r;
        }
        CK(cudaStreamSynchronize(rt->stream));
        for (uint32_t i = 0; i < wave.size(); ++i) {
            if ((wave[i].kind & 0xFFFFu) != kToken) continue;
            IngressEntry *ob = rt->outbox + (size_t)i * rt->outbox_per_msg;
            const uint64_t nout = load_acquire(&ob[0].seq);
            for (uint64_t k = 0; k < nout && k + 1 < rt->outbox_per_msg; ++k) rt->pm_pending.push_back(ob[1 + k]);
        }
    }
    return 0;
}

// Put one message on its way (caller holds rt->mu).
int submit_locked(caf_gpu_runtime *rt, uint32_t a, const caf_gpu_msg *m, uint64_t reply_addr, uint32_t token) {
    if (rt->backend == CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH && (m->kind == kGemmBf16 || m->kind == kGemmSplit)) {
        CK(launch_gemm_one(m->A, m->B, m->C, m->n, m->kind == kGemmSplit, reply_addr, token, rt->d_scratch + 2,
                           rt->cfg.wait_limit_ns, rt->d_ctl, rt->stream));
        rt->launches += 1;
        return 0;
    }
    if (rt->backend == CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH && m->kind == kMandel) {
        const MandelDesc d = *reinterpret_cast<const MandelDesc *>(m->u64);
        CK(launch_mandel_one(d, reply_addr, token, reinterpret_cast<unsigned long long *>(rt->d_scratch + 4),
                             rt->d_scratch + 6, rt->d_ctl, rt->stream));
        rt->launches += 1;
        return 0;
    }
    IngressEntry e{};
    uint64_t payload = m->u64;
    if (m->kind == kMandel) {
        if (!reply_addr) return CAF_GPU_EINVAL;
        const size_t slot = (size_t)((reinterpret_cast<Reply *>(reply_addr)) - rt->replies);
        MandelDesc *d = &rt->mandel_descs[slot];
        *d = *reinterpret_cast<const MandelDesc *>(m->u64);
        payload = (uint64_t)d;
    }
    if (m->kind == kGemmBf16 || m->kind == kGemmSplit) {
        // the drain reads the operands through a descriptor kept with the reply slot
        if (!reply_addr) return CAF_GPU_EINVAL;
        const size_t slot = (size_t)((reinterpret_cast<Reply *>(reply_addr)) - rt->replies);
        GemmDesc *d = &rt->gemm_descs[slot];
        d->A = (uint64_t)m->A;
        d->B = (uint64_t)m->B;
        d->C = (uint64_t)m->C;
        d->n = m->n;
        payload = (uint64_t)d;
    }
    e.actor = a;
    e.kind = m->kind | (m->flags << 16);
    e.sender = m->sender;
    e.sender_seq = rt->sender_seq[m->sender]++;
    e.payload = payload;
    e.reply_addr = reply_addr;
    e.reply_token = token;
    e.tag = m->tag;
    if (rt->backend == CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH) {
        if ((e.kind & 0xFFFFu) == kToken) {
            // token messages may produce more messages: queued, run in waves by
            // caf_gpu_sync / caf_gpu_await
            rt->pm_pending.push_back(e);
            return 0;
        }
        return pm_launch(rt, e, 0);
    }
    const uint32_t cap = rt->cfg.ingress_capacity;
    const uint64_t t = rt->ring_tail;
    if (t - load_acquire(&rt->hctl->ring_consumed) >= cap) {
        int r = kick_locked(rt);
        if (r) return r;
        const uint64_t t0 = now_ns();
        while (t - load_acquire(&rt->hctl->ring_consumed) >= cap) {
            if (rt->hctl->error_word) return device_error(rt->hctl->error_word);
            if (now_ns() - t0 > rt->cfg.wait_limit_ns) return CAF_GPU_EAGAIN;
            kick_locked(rt);
            std::this_thread::yield();
        }
    }
    IngressEntry *slot = &rt->ring[t & (cap - 1)];
    slot->payload = e.payload;
    slot->reply_addr = e.reply_addr;
    slot->tag = e.tag;
    slot->actor = e.actor;
    slot->kind = e.kind;
    slot->sender = e.sender;
    slot->sender_seq = e.sender_seq;
    slot->reply_token = e.reply_token;
    __atomic_store_n(&slot->seq, t + 1, __ATOMIC_RELEASE);
    rt->ring_tail = t + 1;
    return 0;
}

int reserve_reply(caf_gpu_runtime *rt, uint32_t *slot, uint32_t *g) {
    if (rt->free_slots.empty()) return CAF_GPU_EAGAIN;
    *slot = rt->free_slots.back();
    rt->free_slots.pop_back();
    *g = ++rt->gen[*slot];
    if (*g == 0) *g = ++rt->gen[*slot];
    rt->in_use[*slot] = 1;
    rt->replies[*slot].done = 0;
    return 0;
}

void free_runtime(caf_gpu_runtime *rt) {
    if (!rt) return;
    cudaFree(rt->d_ctl);
    cudaFree(rt->d_actors);
    cudaFree(rt->d_slots);
    cudaFree(rt->d_readyq);
    cudaFree(rt->d_freeq);
    cudaFree(rt->d_workq);
    cudaFree(rt->d_packq);
    cudaFree(rt->d_batches);
    cudaFree(rt->d_jobs);
    cudaFree(rt->d_jobq);
    cudaFree(rt->d_jobq_large);
    cudaFree(rt->d_mjobq);
    cudaFree(rt->d_mjobs);
    cudaFree(rt->d_forkq);
    cudaFree(rt->d_segq);
    cudaFree(rt->d_localq_hdr);
    cudaFree(rt->d_localq);
    cudaFree(rt->d_pack_small);
    cudaFree(rt->d_pack_large);
    if (rt->gemm_descs) cudaFreeHost(rt->gemm_descs);
    if (rt->mandel_descs) cudaFreeHost(rt->mandel_descs);
    cudaFree(rt->d_primes);
    cudaFree(rt->d_pinv);
    cudaFree(rt->d_plim);
    cudaFree(rt->d_log);
    cudaFree(rt->d_scratch);
    cudaFree(rt->d_zero);
    if (rt->ring) cudaFreeHost(rt->ring);
    if (rt->hctl) cudaFreeHost(rt->hctl);
    if (rt->replies) cudaFreeHost(rt->replies);
    if (rt->outbox) cudaFreeHost(rt->outbox);
    if (rt->live_done) cudaEventDestroy(rt->live_done);
    if (rt->setup) cudaStreamDestroy(rt->setup);
    if (rt->own_stream && rt->stream) cudaStreamDestroy(rt->stream);
    delete rt;
}

int create_impl(const caf_gpu_runtime_cfg *user, caf_gpu_runtime *rt) {
    caf_gpu_runtime_cfg c{};
    if (user) c = *user;
    if (!c.max_actors) c.max_actors = 16384;
    if (!c.mailbox_capacity) c.mailbox_capacity = 64;
    if (!c.max_inflight_requests) c.max_inflight_requests = 65536;
    if (!c.ingress_capacity) c.ingress_capacity = 65536;
    if (!c.ctas_per_sm) c.ctas_per_sm = 2;
    if (!c.factor_batch) c.factor_batch = 16;
    if (!c.factor_warps) c.factor_warps = 8;
    if (!c.max_factor_n) c.max_factor_n = (1ull << 62) - 1;
    if (!c.mem_budget_bytes) c.mem_budget_bytes = 8ull << 30;
    if (!c.wait_limit_ns) c.wait_limit_ns = 200000000ull;
    if (!c.idle_exit_ns) c.idle_exit_ns = 2000000ull;
    if (!c.log_capacity) c.log_capacity = 1u << 20;
    if (!c.gemm_items_per_round) c.gemm_items_per_round = 4;
    if (!c.fork_pool) c.fork_pool = 1u << 21;
    if (!c.gemm_tile_n) c.gemm_tile_n = 256;
    if (c.gemm_tile_n != 128 && c.gemm_tile_n != 256) return CAF_GPU_EINVAL;
    if (c.scheduler > CAF_GPU_SCHED_STEAL) return CAF_GPU_EINVAL;
    if (c.factor_split > kSplitMax) return CAF_GPU_EINVAL;
    if ((uint64_t)c.max_actors + c.fork_pool >= (1ull << 31)) return CAF_GPU_EINVAL;
    if (c.gemm_items_per_round > kMaxItemsPerRound) return CAF_GPU_EINVAL;
    if (!is_pow2(c.mailbox_capacity) || !is_pow2(c.ingress_capacity)) return CAF_GPU_EINVAL;
    if (c.factor_batch > kFactorKMax || c.ctas_per_sm > 4) return CAF_GPU_EINVAL;
    if (c.factor_warps != 1 && c.factor_warps != 2 && c.factor_warps != 4 && c.factor_warps != 8)
        return CAF_GPU_EINVAL;
    if (c.max_factor_n >= (1ull << 62)) return CAF_GPU_EINVAL;
    if (c.max_actors > (1u << 24)) return CAF_GPU_EINVAL;
    rt->cfg = c;

    CK(cudaGetDevice(&rt->device));
    CK(cudaDeviceGetAttribute(&rt->n_sms, cudaDevAttrMultiProcessorCount, rt->device));
    // every drain CTA must be resident at once (router and ingress warps are
    // waited on by the others), so the grid never exceeds the occupancy limit
    // (with factor_split 0 a launch may run either instantiation: take both)
    int fit = 0, fit_mixed = 0;
    const bool split = c.factor_split > 1;   // launch_drain's instantiation choice
    CK(drain_occupancy(false, split, &fit));
    CK(drain_occupancy(true, split, &fit_mixed));
    if (c.factor_split == 0) {
        int fs = 0, fms = 0;
        CK(drain_occupancy(false, true, &fs));
        CK(drain_occupancy(true, true, &fms));
        fit = std::min(fit, fs);
        fit_mixed = std::min(fit_mixed, fms);
    }
    if (fit < 1 || fit_mixed < 1) return CAF_GPU_ECUDA;
    rt->grid_factor = (unsigned)rt->n_sms * std::min<uint32_t>(c.ctas_per_sm, (uint32_t)fit);
    rt->grid_mixed = (unsigned)rt->n_sms * std::min<uint32_t>(c.ctas_per_sm, (uint32_t)fit_mixed);
    rt->grid = rt->grid_factor;
    if (c.cuda_stream) {
        rt->stream = (cudaStream_t)c.cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&rt->stream, cudaStreamNonBlocking));
        rt->own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&rt->setup, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&rt->live_done, cudaEventDisableTiming));

    // device arena
    CK(cudaMalloc(&rt->d_ctl, sizeof(DevCtl)));
    CK(cudaMemset(rt->d_ctl, 0, sizeof(DevCtl)));
    CK(guarded_malloc(rt, &rt->d_actors, sizeof(ActorDesc) * (size_t)c.max_actors));
    CK(cudaMemset(rt->d_actors, 0, sizeof(ActorDesc) * (size_t)c.max_actors));
    rt->n_slots = (uint64_t)c.max_actors * c.mailbox_capacity;
    CK(guarded_malloc(rt, &rt->d_slots, sizeof(Slot) * rt->n_slots));
    CK(cudaMemset(rt->d_slots, 0, sizeof(Slot) * rt->n_slots));
    rt->n_batches = std::max<uint32_t>(4096, 2u * rt->grid_factor * kConsumerWarps);
    CK(guarded_malloc(rt, &rt->d_batches, sizeof(FactorBatch) * rt->n_batches));
    CK(cudaMemset(rt->d_batches, 0, sizeof(FactorBatch) * rt->n_batches));
    rt->readyq_cap = next_pow2((uint64_t)c.max_actors + 1);
    rt->freeq_cap = next_pow2((uint64_t)rt->n_batches + 1);
    // every job's tiles, or its pack items, can be queued at once
    rt->workq_cap = next_pow2((uint64_t)kGemmJobsSmall * (kPackSmallMaxN / 128) * (kPackSmallMaxN / 128) +
                              (uint64_t)kGemmJobsLarge * (kMaxDrainGemmN / 128) * (kMaxDrainGemmN / 128) +
                              (uint64_t)kMandelJobs * kMandelMaxBands + 1);
    rt->jobq_cap = next_pow2((uint64_t)kGemmJobs + 1);
    std::vector<uint32_t> none, all(rt->n_batches);
    for (uint32_t i = 0; i < rt->n_batches; ++i) all[i] = i;
    int r;
    if ((r = init_queue(rt, &rt->d_readyq, rt->readyq_cap, &rt->d_ctl->readyq, none))) return r;
    if ((r = init_queue(rt, &rt->d_freeq, rt->freeq_cap, &rt->d_ctl->freeq, all))) return r;
    if ((r = init_queue(rt, &rt->d_workq, rt->workq_cap, &rt->d_ctl->workq, none))) return r;
    if ((r = init_queue(rt, &rt->d_packq, next_pow2(2ull * kGemmJobs * (kMaxDrainGemmN / 128) + 1),
                        &rt->d_ctl->packq, none)))
        return r;
    std::vector<uint32_t> jobs_small(kGemmJobsSmall), jobs_large(kGemmJobsLarge);
    for (uint32_t i = 0; i < kGemmJobsSmall; ++i) jobs_small[i] = i;
    for (uint32_t i = 0; i < kGemmJobsLarge; ++i) jobs_large[i] = kGemmJobsSmall + i;
    if ((r = init_queue(rt, &rt->d_jobq, rt->jobq_cap, &rt->d_ctl->jobq, jobs_small))) return r;
    if ((r = init_queue(rt, &rt->d_jobq_large, rt->jobq_cap, &rt->d_ctl->jobq_large, jobs_large))) return r;
    // every batch record split at once still fits
    if ((r = init_queue(rt, &rt->d_segq, (uint32_t)next_pow2((uint64_t)rt->n_batches * kSplitMax + 1),
                        &rt->d_ctl->segq, none)))
        return r;
    CK(guarded_malloc(rt, &rt->d_jobs, sizeof(GemmJob) * kGemmJobs));
    CK(cudaMemset(rt->d_jobs, 0, sizeof(GemmJob) * kGemmJobs));
    std::vector<uint32_t> mjobs(kMandelJobs);
    for (uint32_t i = 0; i < kMandelJobs; ++i) mjobs[i] = i;
    if ((r = init_queue(rt, &rt->d_mjobq, next_pow2((uint64_t)kMandelJobs + 1), &rt->d_ctl->mjobq, mjobs))) return r;
    CK(guarded_malloc(rt, &rt->d_mjobs, sizeof(MandelJob) * kMandelJobs));
    CK(cudaMemset(rt->d_mjobs, 0, sizeof(MandelJob) * kMandelJobs));
    if (c.validation_mode) {
        CK(guarded_malloc(rt, &rt->d_log, sizeof(LogRow) * (size_t)c.log_capacity));
        CK(cudaMemset(rt->d_log, 0, sizeof(LogRow) * (size_t)c.log_capacity));
    }
    if (c.scheduler == CAF_GPU_SCHED_STEAL) {
        // one queue per CTA of the larger grid; cell i of a queue starts free for position i
        const uint32_t nq = std::max(rt->grid_factor, rt->grid_mixed);
        CK(cudaMalloc(&rt->d_localq_hdr, sizeof(QueueHdr) * nq));
        CK(guarded_malloc(rt, &rt->d_localq, sizeof(QCell) * (size_t)nq * kLocalQueueCap));
        std::vector<QueueHdr> hdr(nq);
        for (auto &h : hdr) {
            memset(&h, 0, sizeof(h));
            h.mask = kLocalQueueCap - 1;
        }
        std::vector<QCell> cells((size_t)nq * kLocalQueueCap);
        for (size_t i = 0; i < cells.size(); ++i) {
            cells[i].seq = i % kLocalQueueCap;
            cells[i].val = 0;
            cells[i].pad = 0;
        }
        CK(cudaMemcpy(rt->d_localq_hdr, hdr.data(), sizeof(QueueHdr) * nq, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(rt->d_localq, cells.data(), sizeof(QCell) * cells.size(), cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc(&rt->d_scratch, 64));
    CK(cudaMemset(rt->d_scratch, 0, 64));
    const uint32_t scratch_init[2] = {kNoFactor, 0};
    CK(cudaMemcpy(rt->d_scratch, scratch_init, sizeof(scratch_init), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&rt->d_zero, 64));
    CK(cudaMemset(rt->d_zero, 0, 64));

    // prime table: odd primes up to floor(sqrt(max_factor_n))
    const uint64_t lim = isqrt_u64(c.max_factor_n);
    rt->prime_limit = lim;
    static_assert(kRangePrimes + 64 >= kTile, "the last table tile's copy stays inside the padded table");
    CK(build_prime_table(lim, kRangePrimes + 64, &rt->d_primes, &rt->d_pinv, &rt->d_plim, &rt->nprimes,
                         rt->setup));
    rt->launches += 4;

    // pinned, mapped host memory
    CK(cudaHostAlloc(&rt->ring, sizeof(IngressEntry) * (size_t)c.ingress_capacity, cudaHostAllocMapped));
    memset(rt->ring, 0, sizeof(IngressEntry) * (size_t)c.ingress_capacity);
    CK(cudaHostAlloc(&rt->hctl, sizeof(HostCtl), cudaHostAllocMapped));
    memset(rt->hctl, 0, sizeof(HostCtl));
    CK(cudaHostAlloc(&rt->replies, sizeof(Reply) * (size_t)c.max_inflight_requests, cudaHostAllocMapped));
    memset(rt->replies, 0, sizeof(Reply) * (size_t)c.max_inflight_requests);
    CK(cudaHostAlloc(&rt->gemm_descs, sizeof(GemmDesc) * (size_t)c.max_inflight_requests, cudaHostAllocMapped));
    memset(rt->gemm_descs, 0, sizeof(GemmDesc) * (size_t)c.max_inflight_requests);
    CK(cudaHostAlloc(&rt->mandel_descs, sizeof(MandelDesc) * (size_t)c.max_inflight_requests, cudaHostAllocMapped));
    memset(rt->mandel_descs, 0, sizeof(MandelDesc) * (size_t)c.max_inflight_requests);
    CK(cudaHostAlloc(&rt->outbox, sizeof(IngressEntry) * rt->outbox_per_msg * rt->outbox_msgs,
                     cudaHostAllocMapped));
    memset(rt->outbox, 0, sizeof(IngressEntry) * rt->outbox_per_msg * rt->outbox_msgs);
    rt->free_slots.resize(c.max_inflight_requests);
    for (uint32_t i = 0; i < c.max_inflight_requests; ++i) rt->free_slots[i] = c.max_inflight_requests - 1 - i;
    rt->gen.assign(c.max_inflight_requests, 0);
    rt->in_use.assign(c.max_inflight_requests, 0);
    rt->actors.reserve(1024);
    CK(cudaDeviceSynchronize());
    return 0;
}

// Wait until every host message sent so far has been handled (persistent backend).
int sync_persistent(caf_gpu_runtime *rt) {
    for (;;) {
        {
            std::lock_guard<std::mutex> g(rt->mu);
            int r = kick_locked(rt);
            if (r) return r;
            __atomic_store_n(&rt->hctl->stop, 1u, __ATOMIC_RELEASE);
        }
        CK(cudaStreamSynchronize(rt->stream));
        __atomic_store_n(&rt->hctl->stop, 0u, __ATOMIC_RELEASE);
        if (rt->hctl->error_word) return device_error(rt->hctl->error_word);
        std::lock_guard<std::mutex> g(rt->mu);
        if (load_acquire(&rt->hctl->ring_consumed) == rt->ring_tail) return 0;
    }
}

}  // namespace

extern "C" {

const char *caf_gpu_strerror(int code) {
    switch (code) {
        case CAF_GPU_OK: return "ok";
        case CAF_GPU_EINVAL: return "invalid argument";
        case CAF_GPU_ENOMEM: return "out of memory or table space";
        case CAF_GPU_EAGAIN: return "resource temporarily full, retry";
        case CAF_GPU_ETIMEDOUT: return "timed out";
        case CAF_GPU_EDEAD: return "actor has terminated";
        case CAF_GPU_EWAITLIMIT: return "a bounded device wait expired";
        case CAF_GPU_EBOUNDS: return "validation check: out-of-range index or overwritten guard";
        case CAF_GPU_ESTATE: return "unknown or consumed handle / invalid state";
        case CAF_GPU_ECUDA: return "CUDA error";
        default: return "unknown error";
    }
}

int caf_gpu_runtime_create(const caf_gpu_runtime_cfg *cfg, caf_gpu_runtime **out) {
    if (!out) return CAF_GPU_EINVAL;
    *out = nullptr;
    caf_gpu_runtime *rt = new caf_gpu_runtime();
    int r = create_impl(cfg, rt);
    if (r) {
        free_runtime(rt);
        return r;
    }
    *out = rt;
    return 0;
}

int caf_gpu_runtime_destroy(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    int r = caf_gpu_sync(rt);
    cudaStreamSynchronize(rt->stream);
    const int bad = check_guards(rt);
    free_runtime(rt);
    if (bad > 0) return CAF_GPU_EBOUNDS;
    return (r == CAF_GPU_EWAITLIMIT || r == CAF_GPU_EBOUNDS) ? 0 : r;
}

int caf_gpu_debug_inject(caf_gpu_runtime *rt, uint32_t what, uint64_t arg) {
    if (!rt || rt->capturing) return CAF_GPU_EINVAL;
    int r = caf_gpu_sync(rt);   // no drain runs while a record changes
    if (r) return r;
    std::lock_guard<std::mutex> g(rt->mu);
    if (what == 1) {
        if (!rt->cfg.validation_mode || arg == 0 || arg > rt->n_actors) return CAF_GPU_EINVAL;
        const uint64_t past = rt->n_slots + (uint64_t)kForkSlots * rt->fork_pool;
        CK(cudaMemcpy(&rt->d_actors[arg - 1].slot_base, &past, sizeof(past), cudaMemcpyHostToDevice));
        return 0;
    }
    if (what == 2) {
        if (arg >= rt->guards.size()) return CAF_GPU_EINVAL;
        const uint8_t x = (uint8_t)~kGuardByte;
        CK(cudaMemcpy(rt->guards[arg].second, &x, 1, cudaMemcpyHostToDevice));
        return 0;
    }
    return CAF_GPU_EINVAL;
}

int caf_gpu_check_guards(caf_gpu_runtime *rt, uint32_t *corrupted) {
    if (!rt || !corrupted) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    const int bad = check_guards(rt);
    if (bad < 0) return CAF_GPU_ECUDA;
    *corrupted = (uint32_t)bad;
    return 0;
}

// The FORK actor pool (first FORK spawn): grow the actor table by the pool's
// records and the slot array by their 4-slot mailboxes, copying what exists,
// and fill the free-id queue.  Caller holds rt->mu, and no drain runs.
int make_fork_pool(caf_gpu_runtime *rt) {
    if (rt->graphs_made) return CAF_GPU_ESTATE;   // a graph would keep the old addresses
    const uint32_t pool = rt->cfg.fork_pool;
    const uint32_t base = rt->cfg.max_actors;
    const uint64_t n_act = (uint64_t)base + pool;
    const uint64_t n_slots = rt->n_slots + (uint64_t)kForkSlots * pool;
    ActorDesc *actors = nullptr;
    Slot *slots = nullptr;
    QCell *forkq = nullptr, *readyq = nullptr;
    // on any failure, free what this call made; the runtime keeps its old table
    auto fail_with = [&](int code) {
        cudaGetLastError();
        for (void *p : {(void *)actors, (void *)slots, (void *)forkq, (void *)readyq}) {
            if (p) drop_guard(rt, p);
            cudaFree(p);
        }
        return code;
    };
    if (guarded_malloc(rt, &actors, sizeof(ActorDesc) * n_act) != cudaSuccess) return fail_with(CAF_GPU_ENOMEM);
    if (guarded_malloc(rt, &slots, sizeof(Slot) * n_slots) != cudaSuccess) return fail_with(CAF_GPU_ENOMEM);
    if (cudaMemcpyAsync(actors, rt->d_actors, sizeof(ActorDesc) * base, cudaMemcpyDeviceToDevice, rt->setup) !=
            cudaSuccess ||
        cudaMemcpyAsync(slots, rt->d_slots, sizeof(Slot) * rt->n_slots, cudaMemcpyDeviceToDevice, rt->setup) !=
            cudaSuccess ||
        cudaMemsetAsync(slots + rt->n_slots, 0, sizeof(Slot) * (n_slots - rt->n_slots), rt->setup) != cudaSuccess ||
        launch_fork_pool_init(actors, base, pool, rt->n_slots, rt->setup) != cudaSuccess ||
        cudaStreamSynchronize(rt->setup) != cudaSuccess)
        return fail_with(CAF_GPU_ECUDA);
    // the free-id queue, and a ready queue that holds every actor once (an
    // actor is pushed on the waiting -> ready transition only).  No drain
    // runs, so every actor is parked and the old ready queue is empty.  If the
    // second fails, the first's header is left unused (fork_pool stays 0).
    const uint32_t forkq_cap = (uint32_t)next_pow2((uint64_t)pool + 1);
    const uint32_t readyq_cap = (uint32_t)next_pow2(n_act + 1);
    std::vector<uint32_t> ids(pool);
    for (uint32_t i = 0; i < pool; ++i) ids[i] = base + i;
    int r = init_queue(rt, &forkq, forkq_cap, &rt->d_ctl->forkq, ids);
    if (r) return fail_with(r);
    r = init_queue(rt, &readyq, readyq_cap, &rt->d_ctl->readyq, {});
    if (r) return fail_with(r);
    for (void *p : {(void *)rt->d_readyq, (void *)rt->d_actors, (void *)rt->d_slots}) {
        drop_guard(rt, p);
        cudaFree(p);
    }
    rt->d_readyq = readyq;
    rt->readyq_cap = readyq_cap;
    rt->d_forkq = forkq;
    rt->d_actors = actors;
    rt->d_slots = slots;     // rt->n_slots stays the host actors' region; the pool's slots follow it
    rt->fork_base = base;
    rt->fork_pool = pool;
    return 0;
}

int caf_gpu_spawn(caf_gpu_runtime *rt, uint32_t kernel_id, const caf_gpu_actor_cfg *cfg, caf_gpu_actor *out) {
    if (!rt || !out) return CAF_GPU_EINVAL;
    if (kernel_id < kFactor || kernel_id > kFork) return CAF_GPU_EINVAL;
    const bool recreate = kernel_id == kToken && cfg && (cfg->flags & kActorRecreate);
    if (recreate) {
        // a ring master that creates its ring on the device: its members come
        // from the device actor pool
        if (!(cfg->flags & kActorMaster) || cfg->ring_len < 2 || cfg->ring_len > kRingMaxLen ||
            cfg->incarnations < 1 || cfg->incarnations > kRingMaxIncarnations)
            return CAF_GPU_EINVAL;
        if ((uint64_t)cfg->ring_len - 1 > rt->cfg.fork_pool) return CAF_GPU_EINVAL;
    }
    if (cfg && (cfg->flags & ~(uint32_t)(kActorMaster | kActorRecreate))) return CAF_GPU_EINVAL;
    if ((kernel_id == kFork || recreate) && !rt->fork_pool) {
        int r = caf_gpu_sync(rt);   // stops the running drain: it holds the old table addresses
        if (r) return r;
        std::lock_guard<std::mutex> g(rt->mu);
        if ((r = make_fork_pool(rt))) return r;
    }
    const bool gemm_kind = kernel_id == kGemmBf16 || kernel_id == kGemmSplit;
    if ((gemm_kind && !rt->gemm_enabled) || (kernel_id == kMandel && !rt->mandel_enabled)) {
        // GEMM: drains launched from now on carry the GEMM layout (tensor
        // memory, packs and tiles), and GEMM jobs need their packed-operand
        // scratch.  MANDELBROT: drains launched from now on run work items
        // (in either layout).  Sync first: it stops the running drain, so no
        // drain runs with parameters that predate the actor.
        int r = caf_gpu_sync(rt);
        if (r) return r;
        std::lock_guard<std::mutex> g(rt->mu);
        if (kernel_id == kMandel) rt->mandel_enabled = true;
        if (gemm_kind && !rt->d_pack_small) {
            if (guarded_malloc(rt, &rt->d_pack_small, kPackSmallBytes * kGemmJobsSmall) != cudaSuccess) {
                cudaGetLastError();
                rt->d_pack_small = nullptr;
                return CAF_GPU_ENOMEM;
            }
            if (guarded_malloc(rt, &rt->d_pack_large, kPackLargeBytes * kGemmJobsLarge) != cudaSuccess) {
                cudaGetLastError();
                drop_guard(rt, rt->d_pack_small);
                cudaFree(rt->d_pack_small);
                rt->d_pack_small = rt->d_pack_large = nullptr;
                return CAF_GPU_ENOMEM;
            }
        }
        if (gemm_kind) rt->gemm_enabled = true;
    }
    caf_gpu_actor_cfg c{};
    if (cfg) c = *cfg;
    const uint32_t cap = c.mailbox_capacity ? c.mailbox_capacity : rt->cfg.mailbox_capacity;
    if (!is_pow2(cap) || cap > (1u << 24)) return CAF_GPU_EINVAL;
    std::lock_guard<std::mutex> g(rt->mu);
    if (rt->n_actors >= rt->cfg.max_actors) return CAF_GPU_ENOMEM;
    if (rt->slots_used + cap > rt->n_slots) return CAF_GPU_ENOMEM;
    ActorDesc d{};
    d.kind = kernel_id;
    d.state = kWaiting;
    d.cap_mask = cap - 1;
    d.flags = c.flags;
    d.slot_base = rt->slots_used;
    if (kernel_id == kToken) {
        if (recreate) {
            d.next = kNone;                        // its successor is made on the device
            d.ring_len = c.ring_len;
            d.fork_token = c.incarnations;         // incarnations in all
        } else {
            if (c.next == 0 || c.next > rt->cfg.max_actors) return CAF_GPU_EINVAL;
            d.next = (uint32_t)(c.next - 1);
        }
        if (c.flags & kActorMaster) {
            if (c.worker == 0 || c.worker > rt->n_actors) return CAF_GPU_EINVAL;
            if (rt->actors[c.worker - 1].kind != kFactor) return CAF_GPU_EINVAL;
            d.worker = (uint32_t)(c.worker - 1);
            d.factor_count = c.factor_count;
            d.factor_n = (uint64_t)c.factor_n;
            d.factor_replies = (uint64_t)c.factor_replies;
            if (c.factor_count && (!c.factor_n || !c.factor_replies)) return CAF_GPU_EINVAL;
        }
        d.init_state = c.init_state;
        d.user_state = c.init_state;
    }
    if (kernel_id == kFork) d.next = kNone;   // a root: its answer is the computation's reply
    if (kernel_id == kFactor) ++rt->n_factor_actors;
    if (kernel_id == kSource) {
        // the target must be an existing SINK
        if (c.next == 0 || c.next > rt->n_actors || rt->actors[c.next - 1].kind != kSink) return CAF_GPU_EINVAL;
        d.next = (uint32_t)(c.next - 1);
    }
    const uint32_t idx = rt->n_actors;
    CK(cudaMemcpyAsync(&rt->d_actors[idx], &d, sizeof(d), cudaMemcpyHostToDevice, rt->setup));
    CK(cudaStreamSynchronize(rt->setup));
    rt->slots_used += cap;
    rt->actors.push_back(d);
    rt->n_actors = idx + 1;
    *out = (caf_gpu_actor)idx + 1;
    return 0;
}

int caf_gpu_send(caf_gpu_runtime *rt, caf_gpu_actor to, const caf_gpu_msg *msg) {
    if (rt && rt->capturing) return CAF_GPU_ESTATE;
    uint32_t a;
    int r = check_msg(rt, to, msg, &a);
    if (r) return r;
    // a GEMM or Mandelbrot message needs a reply: its descriptor lives in the reply slot
    if (msg->kind == kGemmBf16 || msg->kind == kGemmSplit || msg->kind == kMandel) return CAF_GPU_EINVAL;
    {
        std::lock_guard<std::mutex> g(rt->mu);
        r = submit_locked(rt, a, msg, 0, 0);
        if (r) return r;
        return kick_locked(rt);
    }
}

int caf_gpu_request(caf_gpu_runtime *rt, caf_gpu_actor to, const caf_gpu_msg *msg, caf_gpu_handle *out) {
    if (rt && rt->capturing) return CAF_GPU_ESTATE;
    if (!out) return CAF_GPU_EINVAL;
    uint32_t a;
    int r = check_msg(rt, to, msg, &a);
    if (r) return r;
    std::lock_guard<std::mutex> g(rt->mu);
    uint32_t slot, gen;
    if ((r = reserve_reply(rt, &slot, &gen))) return r;
    r = submit_locked(rt, a, msg, (uint64_t)&rt->replies[slot], gen);
    if (r) {
        rt->in_use[slot] = 0;
        rt->free_slots.push_back(slot);
        return r;
    }
    *out = ((uint64_t)gen << 32) | (slot + 1);
    return kick_locked(rt);
}

int caf_gpu_request_batch(caf_gpu_runtime *rt, const caf_gpu_actor *to, const caf_gpu_msg *msgs, uint32_t count,
                          caf_gpu_handle *out) {
    if (!rt || (count && (!to || !msgs || !out))) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    for (uint32_t i = 0; i < count; ++i) {
        uint32_t a;
        int r = check_msg(rt, to[i], &msgs[i], &a);
        if (r) return r;
    }
    std::lock_guard<std::mutex> g(rt->mu);
    if (rt->free_slots.size() < count) return CAF_GPU_EAGAIN;
    for (uint32_t i = 0; i < count; ++i) {
        uint32_t slot, gen;
        int r = reserve_reply(rt, &slot, &gen);
        if (r) return r;
        r = submit_locked(rt, (uint32_t)(to[i] - 1), &msgs[i], (uint64_t)&rt->replies[slot], gen);
        if (r) {
            rt->in_use[slot] = 0;
            rt->free_slots.push_back(slot);
            return r;
        }
        out[i] = ((uint64_t)gen << 32) | (slot + 1);
        if ((i & 1023) == 1023) kick_locked(rt);
    }
    return kick_locked(rt);
}

int caf_gpu_await(caf_gpu_runtime *rt, caf_gpu_handle h, uint64_t timeout_ns, caf_gpu_reply *out) {
    if (!rt || !out) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    const uint32_t slot = (uint32_t)(h & 0xFFFFFFFFu) - 1;
    const uint32_t gen = (uint32_t)(h >> 32);
    {
        std::lock_guard<std::mutex> g(rt->mu);
        if (h == 0 || slot >= rt->cfg.max_inflight_requests || !rt->in_use[slot] || rt->gen[slot] != gen)
            return CAF_GPU_ESTATE;
    }
    if (rt->backend == CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH) {
        std::lock_guard<std::mutex> g(rt->mu);
        int r = pm_pump(rt);
        if (r) return r;
    }
    const uint64_t t0 = now_ns();
    uint32_t spins = 0;
    while (load_acquire(&rt->replies[slot].done) != gen) {
        if (const uint32_t w = load_acquire(&rt->hctl->error_word)) return device_error(w);
        if ((++spins & 255) == 0) {
            int r = kick(rt);
            if (r) return r;
            if (rt->backend == CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH && cudaStreamQuery(rt->stream) == cudaSuccess &&
                load_acquire(&rt->replies[slot].done) != gen) {
                // every launch finished and the reply is not there: nothing will write it
                if (timeout_ns && now_ns() - t0 > timeout_ns) return CAF_GPU_ETIMEDOUT;
            }
            if (timeout_ns && now_ns() - t0 > timeout_ns) return CAF_GPU_ETIMEDOUT;
            std::this_thread::yield();
        }
    }
    const Reply &r = rt->replies[slot];
    out->status = r.status;
    out->kind = 0;
    out->r0 = r.r0;
    out->r1 = r.r1;
    out->t_done = r.t_done;
    std::lock_guard<std::mutex> g(rt->mu);
    rt->in_use[slot] = 0;
    rt->free_slots.push_back(slot);
    return 0;
}

int caf_gpu_await_batch(caf_gpu_runtime *rt, const caf_gpu_handle *h, uint32_t count, uint64_t timeout_ns,
                        caf_gpu_reply *out) {
    if (!rt || (count && (!h || !out))) return CAF_GPU_EINVAL;
    for (uint32_t i = 0; i < count; ++i) {
        int r = caf_gpu_await(rt, h[i], timeout_ns, &out[i]);
        if (r) return r;
    }
    return 0;
}

int caf_gpu_request_batch_device(caf_gpu_runtime *rt, const caf_gpu_dmsg *d_msgs, uint32_t count,
                                 caf_gpu_dreply *d_replies) {
    if (!rt || (count && !d_msgs)) return CAF_GPU_EINVAL;
    if (count == 0) return 0;
    std::lock_guard<std::mutex> g(rt->mu);
    if (rt->backend != CAF_GPU_BACKEND_PERSISTENT) return CAF_GPU_ESTATE;
    DrainParams p = make_params(rt);
    p.batch_msgs = d_msgs;
    p.batch_replies = reinterpret_cast<Reply *>(d_replies);
    p.batch_count = count;
    p.n_routers = std::min<uint32_t>(drain_grid(rt) * kConsumerWarps, 128);
    // factor_split 0: a batch smaller than the teams can take (K messages
    // each) leaves teams idle, so it runs the split instantiation, whose idle
    // teams take segments of the large factorizations (factor-only drains;
    // the GEMM layout keeps its one instantiation)
    if (rt->cfg.factor_split == 0 && rt->n_factor_actors && !rt->gemm_enabled) {
        const uint64_t teams = (uint64_t)drain_grid(rt) * (kConsumerWarps / p.factor_w);
        if ((uint64_t)count < teams * rt->cfg.factor_batch) p.split = kSplitMax;
    }
    CK(launch_reset_ctl(rt->d_ctl, rt->stream));
    CK(launch_drain(p, drain_grid(rt), rt->stream));
    rt->launches += 2;
    return 0;
}

int caf_gpu_sync(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    if (rt->backend == CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH) {
        std::lock_guard<std::mutex> g(rt->mu);
        int r = pm_pump(rt);
        if (r) return r;
        CK(cudaStreamSynchronize(rt->stream));
        return 0;
    }
    return sync_persistent(rt);
}

int caf_gpu_stream_sync(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    CK(cudaStreamSynchronize(rt->stream));
    if (rt->hctl->error_word) return device_error(rt->hctl->error_word);
    uint32_t err = 0;
    CK(cudaMemcpy(&err, &rt->d_ctl->error_word, sizeof(err), cudaMemcpyDeviceToHost));
    return err ? device_error(err) : 0;
}

int caf_gpu_set_backend(caf_gpu_runtime *rt, int backend) {
    if (!rt) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    if (backend != CAF_GPU_BACKEND_PERSISTENT && backend != CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH)
        return CAF_GPU_EINVAL;
    int r = caf_gpu_sync(rt);
    if (r) return r;
    std::lock_guard<std::mutex> g(rt->mu);
    rt->backend = backend;
    return 0;
}

int caf_gpu_reset_actors(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    std::lock_guard<std::mutex> g(rt->mu);
    CK(launch_reset_actors(rt->d_actors, rt->n_actors, rt->stream));
    rt->launches += 1;
    return 0;
}

int caf_gpu_actor_state(caf_gpu_runtime *rt, caf_gpu_actor a, uint32_t *lifecycle, int32_t *user_state) {
    if (!rt || a == 0 || a > rt->n_actors) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    ActorDesc d;
    CK(cudaMemcpy(&d, &rt->d_actors[a - 1], sizeof(d), cudaMemcpyDeviceToHost));
    if (lifecycle) *lifecycle = d.state;
    if (user_state) *user_state = d.user_state;
    return 0;
}

int caf_gpu_sink_totals(caf_gpu_runtime *rt, caf_gpu_actor a, uint64_t *count, uint64_t *sum) {
    if (!rt || a == 0 || a > rt->n_actors || rt->actors[a - 1].kind != kSink) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    ActorDesc d;
    CK(cudaMemcpy(&d, &rt->d_actors[a - 1], sizeof(d), cudaMemcpyDeviceToHost));
    if (count) *count = d.sink_count;
    if (sum) *sum = d.sink_sum;
    return 0;
}

int caf_gpu_stats_read(caf_gpu_runtime *rt, caf_gpu_stats *out) {
    if (!rt || !out) return CAF_GPU_EINVAL;
    DevCtl c;
    CK(cudaMemcpy(&c, rt->d_ctl, sizeof(c), cudaMemcpyDeviceToHost));
    const DevCtl &l = rt->last_stats;
    out->launches = rt->launches;
    out->messages = c.messages - l.messages;
    out->device_sends = c.device_sends - l.device_sends;
    out->claims = c.claims - l.claims;
    out->factor_items = c.factor_items - l.factor_items;
    out->prime_tests = c.prime_tests - l.prime_tests;
    out->gemm_tiles = c.gemm_tiles - l.gemm_tiles;
    out->device_spawns = c.device_spawns - l.device_spawns;
    out->error_word = c.error_word;
    out->pad = 0;
    out->diag[0] = c.diag[0];
    out->diag[1] = c.diag[1];
    out->t_mark = c.t_mark;
    rt->last_stats = c;
    rt->launches = 0;
    return 0;
}

int caf_gpu_read_log(caf_gpu_runtime *rt, caf_gpu_log_row *out, uint32_t cap, uint32_t *count) {
    if (!rt || !count) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    if (!rt->d_log) return CAF_GPU_ESTATE;
    CK(cudaStreamSynchronize(rt->stream));
    uint64_t n = 0;
    CK(cudaMemcpy(&n, &rt->d_ctl->log_count, sizeof(n), cudaMemcpyDeviceToHost));
    n = std::min<uint64_t>(n, rt->cfg.log_capacity);
    const uint32_t m = (uint32_t)std::min<uint64_t>(n, cap);
    if (m && out) CK(cudaMemcpy(out, rt->d_log, sizeof(LogRow) * m, cudaMemcpyDeviceToHost));
    const uint64_t zero = 0;
    CK(cudaMemcpy(&rt->d_ctl->log_count, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    *count = m;
    return 0;
}

int caf_gpu_mark(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    std::lock_guard<std::mutex> g(rt->mu);
    CK(launch_mark(rt->d_ctl, rt->stream));
    rt->launches += 1;
    return 0;
}

// ---------------------------------------------------------------------------
// Serving loop
// ---------------------------------------------------------------------------
namespace {

// Ring allocator over the caller's result arena: allocations in admission
// order, space reclaimed from the oldest block once it is freed.
struct ArenaRing {
    uint64_t size = 0, head = 0, tail = 0;     // byte positions modulo size; head - tail in use
    struct Block { uint64_t start, len; bool freed; };
    std::deque<Block> blocks;
    // *off: byte offset in the arena; *id: the block's position (for free_block)
    bool alloc(uint64_t len, uint64_t *off, uint64_t *id) {
        len = (len + 255) & ~255ull;
        if (len > size) return false;
        uint64_t pos = head % size;
        uint64_t skip = 0;
        if (pos + len > size) skip = size - pos;       // do not wrap inside a block
        if (head + skip + len - tail > size) return false;
        if (skip) blocks.push_back({head, skip, true});
        head += skip;
        *off = head % size;
        *id = head;
        blocks.push_back({head, len, false});
        head += len;
        return true;
    }
    // undo the most recent alloc (and its wrap filler)
    void undo_last() {
        if (blocks.empty()) return;
        head = blocks.back().start;
        blocks.pop_back();
        if (!blocks.empty() && blocks.back().freed && blocks.back().start + blocks.back().len == head &&
            head % size == 0) {
            head = blocks.back().start;
            blocks.pop_back();
        }
    }
    void free_block(uint64_t start) {
        for (auto &b : blocks)
            if (b.start == start && !b.freed) {
                b.freed = true;
                break;
            }
        while (!blocks.empty() && blocks.front().freed) {
            tail = blocks.front().start + blocks.front().len;
            blocks.pop_front();
        }
    }
};

struct Inflight {
    uint32_t req, slot, gen;
    uint64_t bytes, arena_start;
    bool gemm;
};

}  // namespace

int caf_gpu_serve_run(caf_gpu_runtime *rt, const caf_gpu_serve_req *reqs, uint32_t count,
                      const caf_gpu_serve_cfg *cfg, caf_gpu_serve_result *results, caf_gpu_serve_stats *stats) {
    if (!rt || (count && (!reqs || !results))) return CAF_GPU_EINVAL;
    if (rt->capturing) return CAF_GPU_ESTATE;
    caf_gpu_serve_cfg c{};
    if (cfg) c = *cfg;
    const uint64_t budget = c.mem_budget_bytes ? c.mem_budget_bytes : rt->cfg.mem_budget_bytes;
    // validate everything before the clock starts
    for (uint32_t i = 0; i < count; ++i) {
        const caf_gpu_serve_req &q = reqs[i];
        if (q.actor == 0 || q.actor > rt->n_actors) return CAF_GPU_EINVAL;
        if (i && q.t_arrival < reqs[i - 1].t_arrival) return CAF_GPU_EINVAL;
        const uint32_t kind = rt->actors[q.actor - 1].kind;
        if (kind == kGemmBf16 || kind == kGemmSplit) {
            if (!q.A || !q.B || q.n == 0 || q.n > kMaxDrainGemmN || !c.c_arena) return CAF_GPU_EINVAL;
            if (12ull * q.n * q.n > budget || 4ull * q.n * q.n > c.c_arena_bytes) return CAF_GPU_EINVAL;
        } else if (kind == kFactor) {
            if (q.u64 > rt->cfg.max_factor_n) return CAF_GPU_EINVAL;
        } else {
            return CAF_GPU_EINVAL;
        }
    }
    int r = caf_gpu_sync(rt);
    if (r) return r;
    ArenaRing arena;
    arena.size = c.c_arena_bytes;
    std::deque<uint32_t> pending;
    std::vector<Inflight> inflight;
    uint64_t inflight_bytes = 0, peak_bytes = 0;
    uint32_t peak_n = 0, next = 0, done = 0;
    const uint64_t launches0 = rt->launches;
    const uint64_t t0 = now_ns();
    auto secs = [&](uint64_t t) { return (double)(t - t0) * 1e-9; };
    while (done < count) {
        const uint64_t now = now_ns();
        if (c.timeout_ns && now - t0 > c.timeout_ns) return CAF_GPU_ETIMEDOUT;
        if (const uint32_t w = load_acquire(&rt->hctl->error_word)) return device_error(w);
        const double tnow = secs(now);
        while (next < count && reqs[next].t_arrival <= tnow) pending.push_back(next++);
        bool progress = false;
        {
            std::lock_guard<std::mutex> g(rt->mu);
            while (!pending.empty()) {
                const uint32_t i = pending.front();
                const caf_gpu_serve_req &q = reqs[i];
                const uint32_t kind = rt->actors[q.actor - 1].kind;
                const bool gemm = kind != kFactor;
                const uint64_t bytes = gemm ? 12ull * q.n * q.n : 0;
                if (inflight_bytes + bytes > budget) break;
                uint64_t off = 0, id = 0;
                if (gemm && !arena.alloc(4ull * q.n * q.n, &off, &id)) break;
                uint32_t slot, gen;
                if (reserve_reply(rt, &slot, &gen)) {
                    if (gemm) arena.undo_last();
                    break;
                }
                caf_gpu_msg m{};
                m.kind = kind;
                m.sender = 0;
                m.u64 = q.u64;
                m.n = q.n;
                m.A = q.A;
                m.B = q.B;
                m.C = gemm ? reinterpret_cast<float *>(static_cast<uint8_t *>(c.c_arena) + off) : nullptr;
                m.tag = i;
                r = submit_locked(rt, q.actor - 1, &m, (uint64_t)&rt->replies[slot], gen);
                if (r) return r;
                results[i].c_offset = off;
                results[i].t_admit = secs(now_ns());
                inflight.push_back({i, slot, gen, bytes, id, gemm});
                inflight_bytes += bytes;
                peak_bytes = std::max(peak_bytes, inflight_bytes);
                peak_n = std::max<uint32_t>(peak_n, (uint32_t)inflight.size());
                pending.pop_front();
                progress = true;
            }
            if (progress) {
                r = kick_locked(rt);
                if (r) return r;
            }
        }
        // completions
        for (size_t k = 0; k < inflight.size();) {
            Inflight &f = inflight[k];
            if (load_acquire(&rt->replies[f.slot].done) == f.gen) {
                const Reply &rep = rt->replies[f.slot];
                caf_gpu_serve_result &res = results[f.req];
                res.status = rep.status;
                res.r0 = rep.r0;
                res.r1 = rep.r1;
                res.t_done = secs(now_ns());
                {
                    std::lock_guard<std::mutex> g(rt->mu);
                    rt->in_use[f.slot] = 0;
                    rt->free_slots.push_back(f.slot);
                }
                inflight_bytes -= f.bytes;
                if (f.gemm) arena.free_block(f.arena_start);
                ++done;
                progress = true;
                f = inflight.back();
                inflight.pop_back();
            } else {
                ++k;
            }
        }
        if (!progress) {
            kick(rt);
            std::this_thread::yield();
        }
    }
    if (stats) {
        stats->wall_s = secs(now_ns());
        stats->peak_inflight_bytes = peak_bytes;
        stats->peak_inflight = peak_n;
        stats->pad = 0;
        stats->launches = rt->launches - launches0;
    }
    return 0;
}

int caf_gpu_graph_begin(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    if (rt->capturing || rt->backend != CAF_GPU_BACKEND_PERSISTENT) return CAF_GPU_ESTATE;
    int r = caf_gpu_sync(rt);   // no live drain may be running on the stream being captured
    if (r) return r;
    std::lock_guard<std::mutex> g(rt->mu);
    CK(cudaStreamBeginCapture(rt->stream, cudaStreamCaptureModeThreadLocal));
    rt->capturing = true;
    return 0;
}

int caf_gpu_graph_end(caf_gpu_runtime *rt, caf_gpu_graph **out) {
    if (!rt || !out) return CAF_GPU_EINVAL;
    std::lock_guard<std::mutex> g(rt->mu);
    if (!rt->capturing) return CAF_GPU_ESTATE;
    rt->capturing = false;
    caf_gpu_graph *gr = new caf_gpu_graph();
    if (cudaStreamEndCapture(rt->stream, &gr->graph) != cudaSuccess ||
        cudaGraphInstantiate(&gr->exec, gr->graph, 0) != cudaSuccess) {
        if (gr->graph) cudaGraphDestroy(gr->graph);
        delete gr;
        return CAF_GPU_ECUDA;
    }
    *out = gr;
    rt->graphs_made = true;
    return 0;
}

int caf_gpu_graph_launch(caf_gpu_runtime *rt, caf_gpu_graph *gr) {
    if (!rt || !gr) return CAF_GPU_EINVAL;
    std::lock_guard<std::mutex> g(rt->mu);
    if (rt->capturing) return CAF_GPU_ESTATE;
    if (live_running(rt)) return CAF_GPU_ESTATE;   // a live drain owns the stream; sync first
    CK(cudaGraphLaunch(gr->exec, rt->stream));
    return 0;
}

int caf_gpu_graph_destroy(caf_gpu_graph *gr) {
    if (!gr) return CAF_GPU_EINVAL;
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
    return 0;
}

void *caf_gpu_stream(caf_gpu_runtime *rt) { return rt ? (void *)rt->stream : nullptr; }

int caf_gpu_prime_table(caf_gpu_runtime *rt, const uint32_t **d_primes, uint32_t *count) {
    if (!rt) return CAF_GPU_EINVAL;
    if (d_primes) *d_primes = rt->d_primes;
    if (count) *count = rt->nprimes;
    return 0;
}

// Test hook: a device wait on a flag that nothing sets must give up after
// `limit_ns` and report CAF_GPU_EWAITLIMIT; the runtime stays usable after
// caf_gpu_clear_error.
int caf_gpu_debug_wait_expiry(caf_gpu_runtime *rt, uint64_t limit_ns) {
    if (!rt) return CAF_GPU_EINVAL;
    CK(launch_debug_wait(rt->d_zero, limit_ns, rt->d_ctl, rt->hctl, rt->stream));
    rt->launches += 1;
    CK(cudaStreamSynchronize(rt->stream));
    return rt->hctl->error_word ? device_error(rt->hctl->error_word) : 0;
}

int caf_gpu_clear_error(caf_gpu_runtime *rt) {
    if (!rt) return CAF_GPU_EINVAL;
    CK(cudaStreamSynchronize(rt->stream));
    const uint32_t zero = 0;
    CK(cudaMemcpy(&rt->d_ctl->error_word, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    rt->hctl->error_word = 0;
    return 0;
}

}  // extern "C"
