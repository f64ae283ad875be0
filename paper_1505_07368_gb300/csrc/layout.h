// Memory layout of the runtime's device-side state, shared by the host
// runtime (which allocates and initialises it) and the kernels.
//
// Everything the drain touches lives in one device arena:
//
//   DevCtl            counters, error word, queue headers      (one per runtime)
//   ActorDesc[A]      actor table, 128 B per actor
//   Slot[S]           mailbox slots, 64 B each; actor a owns a power-of-two
//                     ring of them starting at ActorDesc::slot_base
//   QCell[...]        ready queue (actor ids), free-batch queue, work queue
//   FactorBatch[B]    messages swept together against the prime table
//   GemmJob[272], MandelJob[256]   GEMM / Mandelbrot messages in the drain
//   uint32_t x 3 x P  prime table: odd primes, their inverses mod 2^32 and
//                     floor((2^32-1)/p), structure-of-arrays
//   LogRow[L]         validation-mode handling log
//
// Host-visible state (pinned, mapped) holds the host->device ingress ring,
// the reply slots that caf_gpu_await polls, and a small control block.
#pragma once

#include <cstddef>
#include <cstdint>

namespace cafgpu {

constexpr uint32_t kConsumerWarps = 8;                     // warps that run actors and sweep
constexpr uint32_t kWarpsPerCta = kConsumerWarps + 1;      // + one prime-table producer warp
constexpr uint32_t kThreads = kWarpsPerCta * 32;
constexpr uint32_t kOneThreads = 256;                      // per-message factor kernel
constexpr uint32_t kFactorKMax = 16;     // messages per factor batch, upper bound
constexpr uint32_t kRangePrimes = 4096;  // table padding granule
constexpr uint32_t kNoFactor = 0xFFFFFFFFu;
constexpr uint32_t kTile = 4096;         // primes per staged table tile (128 chunks of 32)
constexpr uint32_t kStages = 2;          // tiles in flight per CTA
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kMaxItemsPerRound = 8;   // GEMM work items a drain CTA may take per round

// One staged tile of the prime table (shared memory, 16-byte aligned).
struct TableTile {
    uint32_t p[kTile];
    uint32_t pinv[kTile];
    uint32_t plim[kTile];
};

// GEMM tile engine geometry (see gemm_tc.cuh): FP32 staging stages of one
// 64-wide k slice each, and a ring of BF16 operand slots of one 16-wide k
// block each.
constexpr uint32_t kGemmF32Stages = 2;
constexpr uint32_t kGemmBfSlots = 6;
constexpr uint32_t kGemmStageBytes = 2u * 128u * 32u * 4u + 64u * 128u * 4u;   // A halves + B: 64 KB
constexpr uint32_t kGemmSlotBytes = 4u * 128u * 16u * 2u;                      // 4 BF16 planes: 16 KB
constexpr uint32_t kPackSlots = 3;         // operand slots of the packed tile loop (drain)
constexpr uint32_t kPackSlotBlocks = 4;    // 16-wide k blocks per packed slot

// Barriers and tensor-memory address of the GEMM tile engine.
struct GemmBars {
    uint64_t f32_full[kGemmF32Stages];     // tensor copies of a staged slice landed
    uint64_t bf_full[kGemmBfSlots];        // converters -> MMA thread (BF16 block ready)
    uint64_t bf_empty[kGemmBfSlots];       // MMA completion -> converters (slot free again)
    uint64_t pk_full[kPackSlots];          // packed tiles: slot's bulk copies landed
    uint64_t pk_empty[kPackSlots];         // packed tiles: slot's MMAs completed
    uint64_t acc_full[2];                  // packed tile sequence: accumulator buffer's MMAs completed
    uint64_t acc_empty[2];                 // packed tile sequence: buffer's epilogue read it (4 warps)
    uint64_t done;                         // last MMA of a tile completed -> epilogue
    uint32_t f32_read[kGemmF32Stages];     // converter warps done with a stage (monotonic count)
    uint32_t tmem;                         // accumulator address from tcgen05.alloc
    uint32_t pad;
};

// A GEMM tile item's job fields, read once (and checked) by the producer lane
// that takes the item.  Every role of the tile run -- bulk copies, MMAs,
// epilogue, the slot and buffer phase counts -- works from this one copy, so
// all of them agree on the tile's geometry.
struct TileSnap {
    uint64_t pack;      // the job record's packed images
    uint64_t C;         // output (n x n, row-major)
    uint32_t n;
    uint32_t tiles;     // the job's tile count: the target of its completion count
    uint16_t tm, tn;    // output tile row, first column panel
    uint8_t split, wide;
    uint16_t pad;
};
static_assert(sizeof(TileSnap) == 32, "TileSnap is 32 bytes");

// Per-CTA shared state of the drain: the table ring's barriers, the GEMM
// barriers, and the group (one factor batch per team of consumer warps).
// The operand area -- table tiles, or GEMM operand tiles -- follows at
// kDrainHeader (1024-byte aligned).
struct GroupShared {
    uint64_t full[kStages];        // producer -> consumers (bulk copies landed)
    uint64_t empty[kStages];       // consumers -> producer (stage free again)
    GemmBars gb;
    uint32_t batch[kConsumerWarps];
    uint32_t limit_tiles;          // tiles needed by the group's largest bound
    uint32_t final_tile;           // tile index at which the group's sequential stream ends
    uint32_t tile_idx[kStages];    // split batches: table tile in each stage (kNone: the stream ended)
    uint32_t active;               // consumer warps still holding messages
    uint32_t exit;
    uint32_t items[kMaxItemsPerRound];   // GEMM work items this CTA runs next
    uint32_t nitems;
    uint32_t mnext;                      // Mandelbrot bands: next 32-pixel group of the round
    unsigned long long msum[kMaxItemsPerRound];   // Mandelbrot bands: escape counts summed
    TileSnap snap[kMaxItemsPerRound];             // GEMM tile items: their job fields (items[i] -> snap[i])
};
constexpr uint32_t kDrainHeader = 1024;
static_assert(sizeof(GroupShared) <= kDrainHeader, "drain header fits");
constexpr uint32_t kTableRingBytes = kStages * (uint32_t)sizeof(TableTile);
// BF16 operand slots + FP32 staging stages
constexpr uint32_t kGemmOpsBytes = kGemmBfSlots * kGemmSlotBytes + kGemmF32Stages * kGemmStageBytes;
// dynamic shared memory of the drain (+1024 for aligning the base)
constexpr uint32_t kDrainSmemFactor = 1024 + kDrainHeader + kTableRingBytes;
constexpr uint32_t kDrainSmemMixed = 1024 + kDrainHeader + (kGemmOpsBytes > kTableRingBytes ? kGemmOpsBytes : kTableRingBytes);

// A GEMM message being computed by the drain: its 128 x 128 output tiles are
// items (job << 16 | tile) in the tile queue.
struct alignas(64) GemmJob {
    uint64_t A, B, C;
    uint32_t n;
    uint32_t split;                // bit 0: split-BF16x3; bit 1: wide tiles (128 x 256, BF16)
    uint32_t tiles;                // tile items of the output
    uint32_t done;                 // tiles finished (atomic)
    uint64_t reply_addr;
    uint32_t reply_token;
    uint32_t packs_left;           // pack items not finished (atomic); the last one queues the tiles
    uint64_t pad;                  // (the record's packed-operand scratch follows from its index)
};
static_assert(sizeof(GemmJob) == 64, "GemmJob is 64 bytes");
constexpr uint32_t kMaxDrainGemmN = 4096;   // <= 1024 tiles per job
// Job records come in two scratch classes: packed operands of a split n x n
// product take 2 ceil(n/128) ceil(n/16) x 8 KB (gemm_packed.cuh), 8 MB for
// n <= 1024 and 128 MB for n <= 4096.
constexpr uint32_t kPackSmallMaxN = 1024;
constexpr uint32_t kGemmJobsSmall = 256;
constexpr uint32_t kGemmJobsLarge = 16;
constexpr uint32_t kGemmJobs = kGemmJobsSmall + kGemmJobsLarge;   // GEMM messages in flight in the drain
constexpr uint64_t kPackSmallBytes = 2ull * 8 * 64 * 8192;       // 8 MB
constexpr uint64_t kPackLargeBytes = 2ull * 32 * 256 * 8192;     // 128 MB

// Operand descriptor referenced by a GEMM message (same layout as caf_gpu_gemm_desc).
struct GemmDesc {
    uint64_t A, B, C;
    uint32_t n;
    uint32_t pad;
};

// Mandelbrot image job (the OpenCL actor experiment of Sec. 5): the pixels of
// rows row0 .. row0+rows-1 of an image `width` wide, pixel (i, j) at
// c = (x0 + i dx) + (y0 + j dy) i; out[(j - row0) * width + i] = its escape
// count.  Same layout as caf_gpu_mandel_desc (40 bytes).
struct MandelDesc {
    uint64_t out;                  // uint32_t counts (device)
    uint32_t width, rows, row0, max_iter;
    float x0, y0, dx, dy;
};
static_assert(sizeof(MandelDesc) == 40, "MandelDesc is 40 bytes");
// A job's band size is chosen at its claim: about two bands per CTA of the
// running grid, within [kMandelBandMin, kMandelBandMax] pixels, a multiple of 32.
constexpr uint32_t kMandelBandMin = 2048;
constexpr uint32_t kMandelBandMax = 8192;
constexpr uint32_t kMandelMaxBands = 2048;           // bands of one job, at most
constexpr uint32_t kMandelMaxPixels = 1u << 24;      // per message
constexpr uint32_t kMandelMaxIter = 1u << 16;        // a band stays well inside the stall limit
constexpr uint32_t kMandelMaxCoord = 1u << 24;       // width and row0 + rows: exact as float32
constexpr uint32_t kMandelJobs = 256;                // Mandelbrot messages in flight in the drain
constexpr uint32_t kMandelItemFlag = 0x4000u;        // work item: band (job << 16 | flag | band)

// A Mandelbrot message being computed by the drain: its bands are items in
// the work queue; the CTA that finishes the last one replies.
struct alignas(64) MandelJob {
    MandelDesc d;
    uint32_t bands;                // band items of the job
    uint32_t done;                 // bands finished (atomic)
    uint64_t sum;                  // escape counts summed so far (atomic)
    uint64_t reply_addr;
    uint32_t reply_token;
    uint32_t band_px;              // pixels per band (a multiple of 32)
};
static_assert(sizeof(MandelJob) == 128, "MandelJob is 128 bytes");
static_assert(kMandelMaxPixels / kMandelBandMax <= kMandelMaxBands, "large jobs fit the band limit");

// actor lifecycle (Sec. 6: ready / waiting / running / done)
enum : uint32_t { kWaiting = 0, kReady = 1, kRunning = 2, kDone = 3 };

// kinds (mirror caf_gpu.h)
enum : uint32_t { kFactor = 1, kGemmBf16 = 2, kGemmSplit = 3, kToken = 4, kSink = 5, kSource = 6, kMandel = 7,
                  kFork = 8 };
enum : uint32_t { kMsgStart = 1, kMsgResult = 2, kMsgRingDone = 4 };
// RECREATE ring masters: at most this many members and incarnations
constexpr uint32_t kRingMaxLen = 1u << 16;
constexpr uint32_t kRingMaxIncarnations = 255;
// FORK: the largest recursion counter (2^n and 2^(n+1) - 2 fit in 32 bits)
constexpr uint32_t kForkMaxN = 30;
constexpr uint32_t kForkSlots = 4;         // mailbox of a pool actor: a start and two results
enum : uint32_t { kActorMaster = 1, kActorRecreate = 2, kActorLink = 4 };

// error codes in DevCtl::error_word (low byte) -- high bits carry the site
enum : uint32_t {
    kErrWaitQueue = 1,     // queue push waited too long
    kErrWaitSlot = 2,      // mailbox slot never published
    kErrWaitSpace = 3,     // mailbox stayed full
    kErrBadMessage = 4,    // device batch named an unknown actor / wrong kind
    kErrDebugWait = 5,     // the debug wait kernel's flag was never set
    kErrGemm = 6,          // GEMM pipeline wait expired
    kErrStall = 7,         // no progress anywhere while messages were in flight
    kErrWaitTable = 8,     // a prime-table bulk copy did not complete
    kErrNoCompletion = 9,  // messages in flight but none completed for kCompletionLimitNs
    kErrBounds = 10,       // validation mode: an index outside its array was refused
};
constexpr uint64_t kCompletionLimitNs = 30ull * 1000 * 1000 * 1000;

// Device-resident message (same layout as caf_gpu_dmsg).
struct caf_dmsg_t {
    uint32_t actor;
    uint32_t kind;
    uint32_t sender;
    uint32_t sender_seq;
    uint64_t u64;
    uint64_t tag;
};
static_assert(sizeof(caf_dmsg_t) == 32, "caf_dmsg_t is 32 bytes");

struct QueueHdr {
    uint64_t enq;                  // tail: next push position
    uint64_t pad0[15];
    uint64_t deq;                  // head: next pop position
    uint64_t pad1[15];
    int64_t avail;                 // published items not yet reserved by a pop
    uint64_t pad3[15];
    uint32_t mask;
    uint32_t pad2[31];
};

struct QCell {
    uint64_t seq;
    uint32_t val;
    uint32_t pad;
};

struct ActorDesc {                 // 128 bytes
    uint32_t kind;
    uint32_t state;                // lifecycle
    uint32_t cap_mask;             // mailbox capacity - 1
    uint32_t flags;
    uint64_t slot_base;            // first Slot of this actor's ring
    uint64_t head;                 // consumer position (written by the claim holder only)
    uint64_t sink_count;           // SINK: messages handled (claim holder only); FORK: actors spawned below;
                                   // RECREATE ring master: the START token each incarnation begins with
    uint64_t sink_sum;             // SINK: sum of their values; FORK: children's results so far
    uint64_t fork_reply;           // FORK root: reply record of the running computation
    uint32_t fork_token;           // FORK root: its reply token; RECREATE ring master: incarnations in all
    uint32_t ring_master;          // ring link (spawned by a RECREATE master): its master
    uint64_t tail;                 // producer ticket (atomic add)
    int32_t user_state;            // TOKEN: last token; FORK: results still awaited
    uint32_t next;                 // TOKEN: ring successor; FORK: parent (kNone for a root)
    uint32_t worker;               // ring master: factor worker
    uint32_t factor_count;         // ring master: number of n values
    uint64_t factor_n;             // ring master: const uint64_t* (device)
    uint64_t factor_replies;       // ring master: reply records (device)
    int32_t init_state;
    uint32_t round;                // ring master: next factor request index
    uint32_t ring_len;             // RECREATE master and its links: actors per ring, master included
    uint32_t ring_pos;             // ring link: its position in the ring (the master is 0)
    uint32_t ring_inc;             // RECREATE master: index of the running incarnation; link: its incarnation
    uint32_t ring_live;            // RECREATE master: members per incarnation while its rings run, else 0
};
static_assert(sizeof(ActorDesc) == 128, "ActorDesc is 128 bytes");

struct Slot {                      // 64 bytes
    uint64_t seq;                  // ticket + 1 once published
    uint64_t payload;              // FACTOR n / TOKEN value / GEMM desc address
    uint64_t reply_addr;           // reply record (0: no reply)
    uint64_t tag;
    uint32_t sender;
    uint32_t sender_seq;
    uint32_t kind;                 // kind | flags << 16
    uint32_t reply_token;          // value stored to the reply's done word
    uint64_t pad[2];
};
static_assert(sizeof(Slot) == 64, "Slot is 64 bytes");
static_assert(offsetof(Slot, reply_addr) % 16 == 0 && offsetof(Slot, sender) % 16 == 0,
              "reply_addr..tag and sender..reply_token are 16-byte vectors");

// Reply record, same layout as caf_gpu_dreply (32 bytes).
struct Reply {
    int32_t status;
    uint32_t done;
    uint64_t r0, r1;
    uint64_t t_done;               // %globaltimer when written
};
static_assert(sizeof(Reply) == 32, "Reply is 32 bytes");

// Host->device ingress entry (64 bytes, pinned memory).
struct IngressEntry {
    uint64_t seq;                  // ticket + 1 once published by the host
    uint64_t payload;
    uint64_t reply_addr;
    uint64_t tag;
    uint32_t actor;
    uint32_t kind;
    uint32_t sender;
    uint32_t sender_seq;
    uint32_t reply_token;
    uint32_t pad[3];
};
static_assert(sizeof(IngressEntry) == 64, "IngressEntry is 64 bytes");

struct FactorBatch {
    uint32_t count;                // messages in the batch
    uint32_t items_left;           // sweeps (team members x segments) not yet finished
    uint32_t maxbound;             // max over messages of pbound
    uint32_t even_mask;            // messages answered by d = 2
    uint64_t n[kFactorKMax];
    uint32_t pbound[kFactorKMax];  // odd primes p in the table with p*p <= n
    uint32_t found[kFactorKMax];   // index of the first dividing prime (atomicMin)
    uint64_t reply_addr[kFactorKMax];
    uint32_t reply_token[kFactorKMax];
    uint64_t tag[kFactorKMax];
    uint32_t segs;                 // segments: segment s sweeps the table tiles i with i % segs == s
    uint32_t pad;
};
// A large batch may be split into segments swept by idle teams in any CTA
// (the factor_split setting); a held batch is (segment << 24) | batch record.
constexpr uint32_t kSplitMax = 32;          // segments of one batch, at most
constexpr uint32_t kSplitMinTiles = 256;    // a batch reaching fewer tiles is not split
constexpr uint32_t kSplitTilesPerSeg = 64;  // at least this many tiles per segment

struct LogRow {                    // same layout as caf_gpu_log_row
    uint32_t actor;
    uint32_t sender;
    uint32_t sender_seq;
    uint32_t kind;
    uint64_t stamp;
    uint64_t tag;
    uint64_t value;
};
static_assert(sizeof(LogRow) == 40, "LogRow is 40 bytes");

struct DevCtl {
    uint64_t ingested;             // messages put into mailboxes (host, batch, device sends)
    uint64_t pad0[15];
    uint64_t completed;            // messages fully handled
    uint64_t pad1[15];
    uint64_t log_count;
    uint64_t ring_head;            // host ring entries taken by the ingress warp
    uint32_t error_word;
    uint32_t exit_flag;
    uint32_t routers_done;
    uint32_t pad2;
    uint64_t heartbeat;            // %globaltimer of the last progress report
    uint64_t diag[2];              // first failure: values seen by the expired wait
    uint64_t t_mark;               // %globaltimer written by k_mark
    // statistics
    uint64_t claims, factor_items, prime_tests, gemm_tiles, device_sends, messages;
    uint64_t device_spawns;        // FORK actors spawned on the device
    uint64_t pad3[4];
    QueueHdr readyq;
    QueueHdr freeq;
    QueueHdr workq;                // GEMM tile items (taken before pack items)
    QueueHdr packq;                // GEMM pack items
    QueueHdr jobq;                 // free GemmJob records, small scratch class
    QueueHdr jobq_large;           // free GemmJob records, large scratch class
    QueueHdr mjobq;                // free MandelJob records
    QueueHdr forkq;                // free ids of the FORK actor pool
    QueueHdr segq;                 // segments of split factor batches, waiting for a team
};

// Host-visible control block (pinned, mapped).
struct HostCtl {
    uint64_t ring_consumed;        // written by the device: ring entries taken
    uint32_t stop;                 // written by the host: leave once quiescent
    uint32_t error_word;           // copy of DevCtl::error_word for the host
    uint32_t pad[12];
};

// Everything a drain launch needs (kernel parameter).
struct DrainParams {
    DevCtl *ctl;
    ActorDesc *actors;
    uint32_t n_actors;
    uint32_t pad0;
    Slot *slots;
    QCell *readyq;
    QCell *freeq;
    QCell *workq;
    QCell *packq;
    FactorBatch *batches;
    const uint32_t *primes;
    const uint32_t *pinv;
    const uint32_t *plim;
    uint32_t nprimes;
    uint32_t factor_k;             // messages per batch (<= kFactorKMax)
    uint32_t factor_w;             // work items per batch
    uint32_t max_claim;            // messages per claim (0: unlimited)
    uint32_t gemm_items;           // GEMM work items per round (1..kMaxItemsPerRound)
    uint32_t pad_gi;
    uint64_t max_n;                // largest factor message accepted
    uint64_t wait_limit_ns;
    uint64_t idle_exit_ns;
    LogRow *log;
    uint32_t log_capacity;
    uint32_t validation;
    // device batch (may be empty)
    const void *batch_msgs;        // caf_gpu_dmsg[count]
    Reply *batch_replies;
    uint32_t batch_count;
    uint32_t n_routers;
    // live host ring (may be absent)
    IngressEntry *ring;
    HostCtl *hctl;
    uint32_t ring_mask;
    uint32_t live;
    // GEMM actors (gemm != 0: tensor memory and the GEMM shared-memory layout)
    GemmJob *jobs;
    QCell *jobq;
    QCell *jobq_large;
    uint8_t *pack_small;           // kGemmJobsSmall x kPackSmallBytes (record j: j-th block)
    uint8_t *pack_large;           // kGemmJobsLarge x kPackLargeBytes (record kGemmJobsSmall + i: i-th)
    uint32_t gemm;
    uint32_t mandel;               // Mandelbrot actors exist: every drain runs work items
    uint32_t gemm_wide;            // BF16 GEMM jobs run 128 x 256 output tiles
    uint32_t pad_gw;
    // Mandelbrot job records
    MandelJob *mjobs;
    QCell *mjobq;
    // FORK actor pool: ids fork_base .. fork_base + fork_pool - 1, free ids in forkq
    QCell *forkq;
    uint32_t fork_base;
    uint32_t fork_pool;
    // work stealing (steal != 0): CTA b's ready queue is localq_hdr[b] with
    // cells localq[b * localq_cap ..]
    QueueHdr *localq_hdr;
    QCell *localq;
    uint32_t localq_cap;
    uint32_t steal;
    // split factor batches (split > 1: at most that many segments per batch)
    QCell *segq;
    uint32_t split;
    uint32_t n_batches;            // batch records (those not in freeq are in use)
    uint64_t n_slots;              // mailbox slots, the pool's included (validation-mode checks)
};
constexpr uint32_t kLocalQueueCap = 4096;     // ready actors per CTA queue
constexpr uint32_t kLocalQueueSlack = 1024;   // room kept for the CTA's concurrent pushes (9 warps x 32 wakes)
constexpr uint32_t kStealTries = 4;           // victims a worker tries per empty pop

}  // namespace cafgpu
