/*
 * caf_gpu.h -- GPU compute actors on one GB300 (sm_103a).
 *
 * Actors live in device memory.  Each has a bounded lock-free mailbox in
 * HBM; a persistent kernel drains the mailboxes, runs the message's
 * data-parallel payload (64-bit trial-division factorization, a dense
 * matrix product on the tcgen05 tensor cores, or a Mandelbrot image), and
 * writes the reply to the request that asked for it.  The calls follow the actor model of
 * "Revisiting Actor Programming in C++" (Charousset, Hiesgen, Schmidt):
 *
 *   caf_gpu_spawn    -- spawn an actor from a compiled-in GPU kernel
 *                       (Sec. 3.6, spawn_cl: an actor facade over a kernel);
 *   caf_gpu_send     -- asynchronous message, no reply (Sec. 4);
 *   caf_gpu_request  -- message with a unique id whose reply is routed back
 *                       to that id only (Sec. 4.3, sync_send);
 *   caf_gpu_await    -- wait for that reply, with an optional timeout
 *                       (Sec. 4.3, ".then" with timeout).
 *
 * All entry points are C, take plain pointers and sizes, and return 0 or a
 * negative CAF_GPU_E* code (caf_gpu_strerror names it).  Nothing here takes
 * or returns a PyTorch type.  Host pointers are ordinary process memory;
 * "device pointer" means memory of the runtime's GPU (cudaMalloc, or a
 * PyTorch CUDA tensor's data pointer).
 *
 * Threading: any host thread may call send/request/await concurrently on
 * one runtime.  Order is kept per (sender, receiver) pair: messages that
 * one sender id sends to one actor are handled in the order sent.
 */
#ifndef CAF_GPU_H
#define CAF_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CAF_GPU_OK          0
#define CAF_GPU_EINVAL     (-1)  /* bad argument, unknown actor, kind mismatch, n out of range */
#define CAF_GPU_ENOMEM     (-2)  /* device memory budget or an internal table is exhausted   */
#define CAF_GPU_EAGAIN     (-3)  /* mailbox / ingress ring / reply table full: back off       */
#define CAF_GPU_ETIMEDOUT  (-4)  /* await timed out; the handle stays valid                   */
#define CAF_GPU_EDEAD      (-5)  /* the receiving actor has terminated                         */
#define CAF_GPU_EWAITLIMIT (-6)  /* a bounded device wait expired; see caf_gpu_error_word      */
#define CAF_GPU_ESTATE     (-7)  /* unknown or already-consumed handle, or runtime misuse      */
#define CAF_GPU_ECUDA      (-8)  /* a CUDA call failed (no GPU, launch failure, ...)           */
#define CAF_GPU_EBOUNDS    (-9)  /* validation: the device refused an out-of-range index, or a */
                                 /* guard region after a device array was overwritten        */

/* ---- kernel ids = message kinds (an actor accepts exactly one kind) ----- */
#define CAF_GPU_FACTOR_U64          1u  /* u64 n -> (p, q), p <= q                   */
#define CAF_GPU_GEMM_BF16           2u  /* C = A*B, BF16 operands, FP32 accumulate   */
#define CAF_GPU_GEMM_SPLIT_BF16X3   3u  /* C = A*B, split-BF16x3 compensated         */
#define CAF_GPU_RING_TOKEN          4u  /* token ring member (stateful)              */
#define CAF_GPU_SINK                5u  /* counts what it receives (stateful)        */
#define CAF_GPU_SOURCE              6u  /* sends a stream of messages to a sink      */
#define CAF_GPU_MANDELBROT          7u  /* escape counts of an image's rows          */
#define CAF_GPU_FORK                8u  /* recursive actor creation (spawns on the device) */
/* SINK and SOURCE are the two ends of the paper's mailbox experiment (Sec. 5,
 * "Mailbox Performance in N:1 Communication Scenario": many senders, one
 * receiver).  A SINK handles each message (u64 value v) by adding 1 to its
 * count and v to its sum (caf_gpu_sink_totals); a request's reply is
 * (count after this message, v).  A SOURCE is spawned with cfg.next = its
 * target SINK; a message u64 = c makes it send c messages to the target, with
 * values (source actor << 32) | k for k = 0 .. c-1, sender = the source, in k
 * order, and a request's reply is (c, 0) once all c are sent.  It sends at most
 * 1024 per run and continues with a message to itself, so a long stream never
 * holds a worker.  Both kinds run in the persistent backend only
 * (CAF_GPU_EINVAL under CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH). */

/* MANDELBROT is the GPU actor of the paper's OpenCL experiment (Sec. 5,
 * "Integrating OpenCL Actors": a 1920 x 1080 Mandelbrot image with 120 or
 * 1200 maximum iterations).  A message names a caf_gpu_mandel_desc: in
 * caf_gpu_msg.u64, the address of one in host memory, copied at the call; in
 * caf_gpu_dmsg.u64, the address of one in device memory, read when the
 * message is handled.  The actor writes the escape count of every pixel of
 * the described rows and replies (r0, r1) = (pixels, sum of the counts).
 * The count of c is the number of updates z <- z^2 + c, from z = 0, made
 * before |z|^2 > 4 is first seen, at most max_iter, with every step one
 * float32 operation rounded to nearest in this order:
 *   x2 = zr*zr; y2 = zi*zi; stop if x2 + y2 > 4;
 *   xy = zr*zi; zi = (xy + xy) + cy; zr = (x2 - y2) + cx;
 * so counts are exact, reproducible integers.  Pixel (i, j) -- column i,
 * image row j -- is c = (x0 + i*dx) + (y0 + j*dy) i, each coordinate one
 * rounded float32 product and sum.  Limits: width * rows <= 2^24,
 * width <= 2^24, row0 + rows <= 2^24, max_iter <= 65536, out 4-byte
 * aligned; other descriptors are EINVAL at the call (host messages) or get
 * reply status CAF_GPU_REPLY_REJECTED (device batches).  A message needs a
 * reply (caf_gpu_send returns EINVAL). */

/* FORK is the actor of the paper's actor-creation benchmark (Sec. 5,
 * "Overhead of Actor Creation": 2^n computed by recursively creating actors).
 * A message u64 = n (0 <= n <= 30) to a FORK actor spawned by the host (the
 * root) starts a computation: an actor with counter c > 0 spawns two FORK
 * actors with counter c - 1 on the device and waits for their results; an
 * actor with counter 0 answers 1; a parent answers the sum of its two
 * children's results and terminates.  The root's reply is (r0, r1) =
 * (2^n, actors spawned = 2^(n+1) - 2).  Spawned actors come from a device
 * pool of cfg.fork_pool actor records (made at the first FORK spawn); a
 * terminated actor's record returns to the pool, so repeated computations
 * recycle the same records.  A message is EINVAL at the call (REJECTED in a
 * device batch) when its tree, 2^(n+1) - 2 actors, exceeds the pool; the
 * trees in flight at once share the pool, and a spawn that finds it empty
 * waits, bounded by wait_limit_ns (then CAF_GPU_EWAITLIMIT).  A root handles
 * one computation at a time: a start message that reaches it while it waits
 * for results gets CAF_GPU_REPLY_REJECTED.  Spawn the first FORK actor before
 * recording any CUDA graph (ESTATE after one): making the pool moves the
 * actor table.  Persistent backend only. */

/* ---- backends ----------------------------------------------------------- */
#define CAF_GPU_BACKEND_PERSISTENT          0  /* one persistent kernel drains all mailboxes */
#define CAF_GPU_BACKEND_PER_MESSAGE_LAUNCH  1  /* one kernel launch per message (comparator)  */

/* ---- schedulers (Sec. 6.2) ------------------------------------------------ */
#define CAF_GPU_SCHED_GLOBAL  0u   /* one device-wide queue of ready actors                      */
#define CAF_GPU_SCHED_STEAL   1u   /* a queue per worker CTA: the actors a CTA wakes go to its    */
                                   /* own queue; an idle CTA steals from others (work stealing)  */

/* ---- reply status ------------------------------------------------------- */
#define CAF_GPU_REPLY_OK        0  /* factor: n = r0 * r1 with r0 the smallest divisor >= 2 */
#define CAF_GPU_REPLY_NOFACTOR  1  /* factor: no divisor d >= 2 with d*d <= n; (r0, r1) = (1, n) */
#define CAF_GPU_REPLY_DEAD      2  /* the receiver had terminated; nothing was computed     */
#define CAF_GPU_REPLY_REJECTED  3  /* device batch: unknown actor, kind mismatch or n too big */

/* ---- message flags ------------------------------------------------------ */
#define CAF_GPU_MSG_START  0x1u    /* RING_TOKEN: start the ring at this master   */

/* ---- actor flags -------------------------------------------------------- */
#define CAF_GPU_ACTOR_MASTER   1u    /* RING_TOKEN: ring master (emits factor requests)          */
#define CAF_GPU_ACTOR_RECREATE 2u    /* RING_TOKEN master: creates its ring on the device, anew  */
                                     /* for each of cfg.incarnations runs (see below)            */
/* A re-creating ring master (MASTER | RECREATE) is the paper's mixed-benchmark
 * ring master whose ring "is re-created 4 times" (Sec. 5, "Mixed Operations
 * Under Work Load").  It is spawned by the host with cfg.ring_len (actors per
 * ring, master included, 2..65536), cfg.incarnations (1..255), its factor
 * worker and factor arrays; cfg.next is ignored.  A START message with token
 * v makes it spawn ring_len - 1 member actors on the device (from the FORK
 * actor pool, made at this spawn if absent), run the ring with token v, and,
 * when every member has terminated, spawn the next incarnation's members,
 * until cfg.incarnations have run; then it terminates.  Members terminate as
 * in a plain ring and their records return to the pool.  Factor requests go
 * out at each incarnation's start and per token v > 0 the master receives
 * (factor_count must cover them all).  A START that reaches a master whose
 * ring is running gets CAF_GPU_REPLY_REJECTED.  Spawn it before recording any
 * CUDA graph (ESTATE after one).  Persistent backend only.  Token values are
 * at most 2^31 - 1. */

typedef struct caf_gpu_runtime caf_gpu_runtime;   /* opaque */
typedef uint64_t caf_gpu_actor;                   /* opaque actor id, 0 = invalid */
typedef uint64_t caf_gpu_handle;                  /* request handle, 0 = invalid  */

/*
 * Runtime configuration (the scheduler knobs of Sec. 6.1, set_scheduler:
 * number of workers and maximum messages per actor run).  Zero selects the
 * default named after each field.
 */
typedef struct {
    uint32_t max_actors;            /* actor table size (default 16384)                       */
    uint32_t mailbox_capacity;      /* default mailbox slots per actor, power of two (64)     */
    uint32_t max_inflight_requests; /* host reply slots (default 65536)                       */
    uint32_t ingress_capacity;      /* host->device ring slots, power of two (65536)          */
    uint32_t ctas_per_sm;           /* persistent CTAs per SM: the worker count (default 2)   */
    uint32_t max_msgs_per_claim;    /* messages one claim of an actor may take; 0 = no limit  */
                                    /* (GEMM claims ignore it and take up to 32)              */
    uint32_t factor_batch;          /* messages swept together as one batch (<= 16, default 16) */
    uint32_t factor_warps;          /* warps sharing one batch: 1, 2, 4 or 8 (default 8); 1   */
                                    /* while no FACTOR actor exists (every warp claims actors) */
    uint64_t max_factor_n;          /* largest accepted n, < 2^62 (default 2^62 - 1)          */
    uint64_t mem_budget_bytes;      /* serving admission budget (default 8 GiB)               */
    uint64_t wait_limit_ns;         /* every device spin-wait gives up after this (200 ms)    */
    uint64_t idle_exit_ns;          /* persistent kernel exits after this idle time (2 ms)    */
    uint32_t validation_mode;       /* 1: record a handling log (caf_gpu_read_log)            */
    uint32_t log_capacity;          /* log rows (default 1 << 20)                             */
    void    *cuda_stream;           /* cudaStream_t for all work; NULL = runtime's own stream */
    uint32_t gemm_items_per_round;  /* GEMM work items a drain CTA takes per round, 1..8 (4)   */
    uint32_t fork_pool;             /* FORK actors the device may hold at once (2^21)          */
    uint32_t scheduler;             /* ready actors: CAF_GPU_SCHED_* (global queue)            */
    uint32_t factor_split;          /* S > 1: a large factor batch is split into up to S       */
                                    /* (<= 32) segments that idle teams in other CTAs sweep;   */
                                    /* 1: never split; 0 (default): a device batch with fewer  */
                                    /* messages than the drain's teams take (K each) splits    */
                                    /* with S = 32, other launches do not split                */
    uint32_t gemm_tile_n;           /* GEMM_BF16 output tile width in the drain: 128 or 256    */
                                    /* (default 256; split-BF16x3 always uses 128)              */
} caf_gpu_runtime_cfg;

/* Per-actor configuration for caf_gpu_spawn (may be NULL for defaults). */
typedef struct {
    uint32_t mailbox_capacity;      /* power of two; 0 = runtime default                       */
    uint32_t flags;                 /* CAF_GPU_ACTOR_*                                         */
    caf_gpu_actor next;             /* RING_TOKEN: successor in the ring                       */
    caf_gpu_actor worker;           /* RING_TOKEN master: its factorization worker             */
    int32_t  init_state;            /* RING_TOKEN: initial user state (0)                      */
    uint32_t factor_count;          /* RING_TOKEN master: entries in factor_n                  */
    const uint64_t *factor_n;       /* RING_TOKEN master: device array, n sent at round k      */
    void *factor_replies;           /* RING_TOKEN master: device caf_gpu_dreply[factor_count]  */
    uint32_t ring_len;              /* RECREATE master: actors per ring, master included       */
    uint32_t incarnations;          /* RECREATE master: rings it creates, one after another    */
} caf_gpu_actor_cfg;

/* A message.  Copied at the call (call-by-value, Sec. 3.3); GEMM operands
 * are borrowed: A and B read-only, C written, all device pointers that must
 * stay valid until the reply has been awaited (or caf_gpu_sync returned). */
typedef struct {
    uint32_t kind;                  /* CAF_GPU_* kernel id; must equal the actor's             */
    uint32_t flags;                 /* CAF_GPU_MSG_*                                           */
    uint32_t sender;                /* sender id: order is kept per (sender, receiver)         */
    uint32_t n;                     /* GEMM: matrix size (n x n, row-major, leading dim n)     */
    uint64_t u64;                   /* FACTOR_U64: the number; RING_TOKEN: the token value;    */
                                    /* MANDELBROT: address of a host caf_gpu_mandel_desc       */
    uint64_t tag;                   /* caller's tag, echoed in the handling log                */
    const float *A;                 /* GEMM operands (device)                                  */
    const float *B;
    float *C;                       /* GEMM result (device)                                    */
} caf_gpu_msg;

/* A reply. */
typedef struct {
    int32_t  status;                /* CAF_GPU_REPLY_*                                         */
    uint32_t kind;
    uint64_t r0, r1;                /* FACTOR_U64: (p, q) with p <= q; GEMM: (0, n);           */
                                    /* MANDELBROT: (pixels, sum of the escape counts);         */
                                    /* FORK: (2^n, actors spawned)                             */
    uint64_t t_done;                /* device clock when the reply was written (ns)            */
} caf_gpu_reply;

/* Device-resident message for caf_gpu_request_batch_device (32 bytes). */
typedef struct {
    uint32_t actor;                 /* actor index: the caf_gpu_actor value minus one          */
    uint32_t kind;                  /* kernel id | (CAF_GPU_MSG_* << 16)                       */
    uint32_t sender;
    uint32_t sender_seq;            /* position in that sender's stream (for the log)          */
    uint64_t u64;                   /* FACTOR: n; TOKEN: value; GEMM: device address of a      */
                                    /* caf_gpu_gemm_desc; MANDELBROT: device address of a      */
                                    /* caf_gpu_mandel_desc                                      */
    uint64_t tag;
} caf_gpu_dmsg;

/* GEMM operand descriptor referenced by a caf_gpu_dmsg (device memory, 32 bytes). */
typedef struct {
    const float *A;
    const float *B;
    float *C;
    uint32_t n;
    uint32_t pad;
} caf_gpu_gemm_desc;

/* Mandelbrot job referenced by a MANDELBROT message (40 bytes).  out is device
 * memory of width * rows uint32 counts, row-major: out[(j - row0) * width + i]
 * is pixel (i, j); the caller owns it, and it must stay valid until the reply
 * has been awaited. */
typedef struct {
    uint32_t *out;
    uint32_t width;                 /* pixels per row                                          */
    uint32_t rows;                  /* rows in this job                                        */
    uint32_t row0;                  /* image row index j of the first row                      */
    uint32_t max_iter;              /* iteration limit (<= 65536)                              */
    float x0, y0;                   /* c of pixel (0, 0) of the image                          */
    float dx, dy;                   /* step of c per column and per row                        */
} caf_gpu_mandel_desc;

/* Device-resident reply written by the drain (32 bytes). */
typedef struct {
    int32_t  status;                /* CAF_GPU_REPLY_*                                         */
    uint32_t done;                  /* 1 once written                                          */
    uint64_t r0, r1;
    uint64_t t_done;                /* device clock (%globaltimer, ns) when the reply was written */
} caf_gpu_dreply;

/* One row of the validation-mode handling log. */
typedef struct {
    uint32_t actor;                 /* handling actor                                           */
    uint32_t sender;
    uint32_t sender_seq;
    uint32_t kind;                  /* kind | flags << 16                                       */
    uint64_t stamp;                 /* increases with handling order                            */
    uint64_t tag;
    uint64_t value;                 /* FACTOR: n; TOKEN: token value                            */
} caf_gpu_log_row;

/* Counters of the most recent drain. */
typedef struct {
    uint64_t launches;              /* kernels the runtime has launched                         */
    uint64_t messages;              /* messages handled                                         */
    uint64_t device_sends;          /* messages sent by actors on the device                    */
    uint64_t claims;                /* actor claims                                             */
    uint64_t factor_items;          /* factor work items run                                    */
    uint64_t prime_tests;           /* (prime, n) divisibility tests run                        */
    uint64_t gemm_tiles;            /* GEMM output tiles computed                               */
    uint32_t error_word;            /* nonzero: a bounded wait expired (code | site << 8)      */
    uint32_t pad;
    uint64_t diag[2];               /* values the expired wait saw (for diagnosis)              */
    uint64_t t_mark;                /* device clock of the last caf_gpu_mark (ns)               */
    uint64_t device_spawns;         /* FORK actors spawned on the device                        */
} caf_gpu_stats;

/* Create a runtime on the current CUDA device.  Builds the prime table used by
 * FACTOR_U64 actors (odd primes up to floor(sqrt(max_factor_n))).  `cfg` may be
 * NULL.  Errors: EINVAL (bad cfg), ENOMEM, ECUDA. */
int caf_gpu_runtime_create(const caf_gpu_runtime_cfg *cfg, caf_gpu_runtime **out);

/* Drain outstanding work, stop the kernel and free everything.  Unawaited
 * handles become invalid. */
int caf_gpu_runtime_destroy(caf_gpu_runtime *rt);

/* Spawn an actor that runs compiled-in kernel `kernel_id` (Sec. 3.6 spawn_cl:
 * the kernel is fixed at spawn, the message carries the arguments).  No kernel
 * launch.  Errors: EINVAL (unknown kernel id, bad cfg), ENOMEM (actor table or
 * mailbox pool full). */
int caf_gpu_spawn(caf_gpu_runtime *rt, uint32_t kernel_id, const caf_gpu_actor_cfg *cfg,
                  caf_gpu_actor *out);

/* Asynchronous send (no reply).  EINVAL if msg->kind differs from the actor's
 * kernel id (the runtime form of the paper's compile-time interface check,
 * Sec. 4.3); EDEAD if the actor has terminated; EAGAIN if the ingress ring is full. */
int caf_gpu_send(caf_gpu_runtime *rt, caf_gpu_actor to, const caf_gpu_msg *msg);

/* Request: like send, but assigns a unique request id and reserves a reply
 * slot; the reply goes to that id only (Sec. 4.3).  EAGAIN if no reply slot is free. */
int caf_gpu_request(caf_gpu_runtime *rt, caf_gpu_actor to, const caf_gpu_msg *msg,
                    caf_gpu_handle *out);

/* Wait until the reply of `h` arrives, or `timeout_ns` passes (0 = wait
 * forever).  On success copies it to *out and frees the handle.  ETIMEDOUT
 * leaves the handle valid; ESTATE for an unknown or consumed handle;
 * EWAITLIMIT if the device gave up a bounded wait. */
int caf_gpu_await(caf_gpu_runtime *rt, caf_gpu_handle h, uint64_t timeout_ns,
                  caf_gpu_reply *out);

/* Batched host forms: `count` requests / awaits in one call (same semantics as
 * the single calls, in array order; sender order is array order). */
int caf_gpu_request_batch(caf_gpu_runtime *rt, const caf_gpu_actor *to, const caf_gpu_msg *msgs,
                          uint32_t count, caf_gpu_handle *out);
int caf_gpu_await_batch(caf_gpu_runtime *rt, const caf_gpu_handle *h, uint32_t count,
                        uint64_t timeout_ns, caf_gpu_reply *out);

/* Device-resident batch: `count` messages at device address `d_msgs`; the
 * reply of message i is written to d_replies[i] (device).  Enqueued on the
 * runtime stream, in stream order; it returns at once and the replies are
 * complete when the stream reaches this point (caf_gpu_stream_sync).  Order per
 * (sender, actor) is array order.  The kinds are checked on the device: a
 * message whose kind does not match its actor, or whose actor is unknown or
 * terminated, is not handled and gets reply status CAF_GPU_REPLY_DEAD. */
int caf_gpu_request_batch_device(caf_gpu_runtime *rt, const caf_gpu_dmsg *d_msgs, uint32_t count,
                                 caf_gpu_dreply *d_replies);

/* Process everything sent so far and wait for it (both backends). */
int caf_gpu_sync(caf_gpu_runtime *rt);

/* Wait for the runtime stream. */
int caf_gpu_stream_sync(caf_gpu_runtime *rt);

/* Select the backend for subsequent messages (only while nothing is in flight). */
int caf_gpu_set_backend(caf_gpu_runtime *rt, int backend);

/* Reset every RING_TOKEN actor to its spawn state (lifecycle and user state)
 * and zero every SINK's totals, stream-ordered, so a workload can be replayed
 * or captured in a CUDA graph. */
int caf_gpu_reset_actors(caf_gpu_runtime *rt);

/* Lifecycle (0 waiting, 1 ready, 2 running, 3 done) and user state of an actor. */
int caf_gpu_actor_state(caf_gpu_runtime *rt, caf_gpu_actor a, uint32_t *lifecycle,
                        int32_t *user_state);

/* A SINK's totals: messages handled and the sum of their values.  EINVAL if
 * `a` is not a SINK. */
int caf_gpu_sink_totals(caf_gpu_runtime *rt, caf_gpu_actor a, uint64_t *count, uint64_t *sum);

/* Counters and the device error word since the last call (which resets them). */
int caf_gpu_stats_read(caf_gpu_runtime *rt, caf_gpu_stats *out);

/* Copy up to `cap` rows of the validation-mode handling log and clear it. */
int caf_gpu_read_log(caf_gpu_runtime *rt, caf_gpu_log_row *out, uint32_t cap, uint32_t *count);

/* Record the device clock (%globaltimer, ns) on the runtime stream, in stream
 * order; caf_gpu_stats_read returns it as t_mark.  Replies carry the same
 * clock in t_done, so t_done - t_mark is a message's latency from the mark. */
int caf_gpu_mark(caf_gpu_runtime *rt);

/* ---- CUDA graphs -----------------------------------------------------------
 * The stream-ordered calls -- caf_gpu_reset_actors, caf_gpu_request_batch_device,
 * caf_gpu_mark -- can be recorded once into a CUDA graph and replayed with one
 * launch, so a whole actor workload (for example: reset the rings, send each
 * master its start message, drain to completion) costs one host call.  The
 * paper has no counterpart; it is how this library batches whole workloads.
 * Between begin and end those calls are recorded, not run; every call that
 * waits for the device (send, request, await, sync, stream_sync, read_log,
 * actor_state) returns CAF_GPU_ESTATE.  The device buffers a recorded call
 * names must stay valid while the graph exists. */
typedef struct caf_gpu_graph caf_gpu_graph;   /* opaque */
int caf_gpu_graph_begin(caf_gpu_runtime *rt);
int caf_gpu_graph_end(caf_gpu_runtime *rt, caf_gpu_graph **out);
/* Launch the graph on the runtime stream (returns at once; caf_gpu_stream_sync waits). */
int caf_gpu_graph_launch(caf_gpu_runtime *rt, caf_gpu_graph *g);
int caf_gpu_graph_destroy(caf_gpu_graph *g);

/* The runtime's CUDA stream (cudaStream_t). */
void *caf_gpu_stream(caf_gpu_runtime *rt);

/* Number of odd primes in the runtime's prime table and a device pointer to
 * them (uint32_t, increasing). */
int caf_gpu_prime_table(caf_gpu_runtime *rt, const uint32_t **d_primes, uint32_t *count);

/* Fault-path test hook: launch a kernel whose bounded wait on a flag that
 * nothing sets must give up after `limit_ns`.  Returns CAF_GPU_EWAITLIMIT when
 * the expiry was reported through the error word (the expected result); no
 * fault, trap or hang is involved.  caf_gpu_clear_error makes the runtime
 * usable again. */
int caf_gpu_debug_wait_expiry(caf_gpu_runtime *rt, uint64_t limit_ns);

/* Measured throughput, on the current device, of the 32-bit multiplies the
 * factorization test is built from (the test is two low multiplies and one
 * high multiply per (n, p) pair; Sec. 5's prime factorization, see
 * caf_gpu_spawn): rates[0] = low multiply-adds/s, rates[1] = high multiplies/s,
 * rates[2] = multiplies/s of the test's own three-multiply chain.  rates:
 * host array of 3 doubles.  Runs three short kernels (a few ms) on the
 * current device and allocates, then frees, a small buffer; needs no runtime.
 * Returns CAF_GPU_EINVAL for a null pointer, CAF_GPU_ECUDA on a CUDA error. */
int caf_gpu_measure_mul_rates(double *rates);

/* Measured throughput, on the current device, of float32 multiplies and adds
 * (each rounded on its own, no fused multiply-add): the operations of the
 * MANDELBROT escape iteration.  *ops_per_s = operations per second over all
 * SMs.  Runs two short kernels on the current device and allocates, then
 * frees, a small buffer; needs no runtime.  CAF_GPU_EINVAL for a null
 * pointer, CAF_GPU_ECUDA on a CUDA error. */
int caf_gpu_measure_fp32_rate(double *ops_per_s);

/* Measured latencies, on the current device, of the memory operations a
 * mailbox hop is built from (a token passed along a ring of actors, Sec. 5,
 * "Mixed Operations Under Work Load", is a chain of such dependent steps):
 * ns[0] = a returning atomic add (dependent chain, one thread: one L2 round
 * trip), ns[1] = an acquire load of a line held in L2 (dependent chain),
 * ns[2] = a relaxed store followed by fence.sc.gpu, ns[3] = a one-way flag
 * handoff between two SMs (release store, acquire polling; half a ping-pong
 * round trip).  ns: host array of 4 doubles.  Runs two short kernels on the
 * current device (the ping-pong as a cooperative launch of two CTAs on two
 * SMs, every wait bounded) and allocates, then frees, small buffers; needs no
 * runtime.  CAF_GPU_EINVAL for a null pointer, CAF_GPU_ECUDA on a CUDA error
 * or a wait that gave up. */
int caf_gpu_measure_latency(double *ns);

/* Arena canaries.  Every device array of the runtime is followed by a guard
 * region that no kernel writes; this call reads them all back and sets
 * *corrupted to the number whose bytes changed (0 when memory is intact).  The
 * same check runs in caf_gpu_runtime_destroy, which then returns
 * CAF_GPU_EBOUNDS.  Not while recording a graph (ESTATE).  The paper has no
 * counterpart: it is the library's own memory-safety check. */
int caf_gpu_check_guards(caf_gpu_runtime *rt, uint32_t *corrupted);

/* Fault-injection test hook, host side only (no device fault is made):
 * what = 1: point the mailbox of actor `arg` (a caf_gpu_actor) past the end of
 * the slot pool; the next message to it must be refused by the validation-mode
 * bounds check (CAF_GPU_EBOUNDS from the call that waits for it), with nothing
 * read or written out of range.  Needs validation_mode (EINVAL otherwise); the
 * actor stays unusable.  what = 2: overwrite one byte of guard region `arg`
 * (0-based), which caf_gpu_check_guards then reports.  EINVAL for anything
 * else. */
int caf_gpu_debug_inject(caf_gpu_runtime *rt, uint32_t what, uint64_t arg);

/* Clear the device error word after a reported bounded-wait expiry. */
int caf_gpu_clear_error(caf_gpu_runtime *rt);

/* ---- serving loop ---------------------------------------------------------
 * Open-loop serving with continuous batching.  Requests arrive at their
 * t_arrival (seconds from the start of the run, non-decreasing); a request
 * is admitted, in arrival order, once the bytes of the requests in flight
 * plus its own fit the memory budget (GEMM: 12 n^2 bytes for A, B and C;
 * factorization: 0) and its result buffer can be placed in the caller's
 * result arena.  Admitted requests go to the running drain at once, so new
 * work overlaps work already on the GPU; memory and reply slots are released
 * as replies arrive.  The paper has no serving experiment; this is the
 * measurement harness of the library, in the library so its timestamps are
 * taken next to the calls they time.
 *
 * Ownership: reqs, results and stats are host arrays owned by the caller.
 * GEMM operands A and B are the caller's device matrices, borrowed for the
 * run; each GEMM result is written into c_arena (caller's device memory) at
 * results[i].c_offset (bytes) and stays there until the next run. */
typedef struct {
    caf_gpu_actor actor;            /* receiver (its kind is the request kind)                */
    double   t_arrival;             /* seconds from the start of the run                      */
    uint64_t u64;                   /* FACTOR_U64: n                                          */
    uint32_t n;                     /* GEMM: matrix size                                      */
    uint32_t pad;
    const float *A;                 /* GEMM operands (device), n x n row-major                */
    const float *B;
} caf_gpu_serve_req;

typedef struct {
    int32_t  status;                /* reply status                                            */
    uint32_t pad;
    uint64_t r0, r1;                /* reply values                                            */
    uint64_t c_offset;              /* GEMM: byte offset of C in c_arena                       */
    double   t_admit;               /* seconds from the start: admitted and sent               */
    double   t_done;                /* seconds from the start: reply seen by the host          */
} caf_gpu_serve_result;

typedef struct {
    uint64_t mem_budget_bytes;      /* 0: the runtime's mem_budget_bytes                      */
    void    *c_arena;               /* device memory for GEMM results                         */
    uint64_t c_arena_bytes;
    uint64_t timeout_ns;            /* give up (ETIMEDOUT) after this long; 0 = no limit      */
} caf_gpu_serve_cfg;

typedef struct {
    double   wall_s;                /* first arrival to last reply                             */
    uint64_t peak_inflight_bytes;   /* never above the budget                                  */
    uint32_t peak_inflight;         /* requests in flight at most                              */
    uint32_t pad;
    uint64_t launches;              /* kernels launched by the runtime during the run          */
} caf_gpu_serve_stats;

int caf_gpu_serve_run(caf_gpu_runtime *rt, const caf_gpu_serve_req *reqs, uint32_t count,
                      const caf_gpu_serve_cfg *cfg, caf_gpu_serve_result *results,
                      caf_gpu_serve_stats *stats);

/* ---- factorization without device allocation ----------------------------
 *
 * The paper has no counterpart to this call: it exists for callers of this
 * library that cannot call cudaMalloc -- code inside a host framework whose
 * allocator owns the GPU's memory, latency-critical paths that cannot take
 * cudaMalloc's device-wide synchronisation, programs that forbid dynamic
 * allocation after start-up.  Such callers cannot create a runtime (it
 * allocates), so this call needs none.
 *
 * Factors d_n[0..count) (device memory) and writes reply i to d_replies[i]
 * (device memory): status CAF_GPU_REPLY_OK with (r0, r1) = (smallest divisor
 * d >= 2 with d*d <= n, n/d), CAF_GPU_REPLY_NOFACTOR with (1, n), or
 * CAF_GPU_REPLY_REJECTED for n >= 2^62.  The results equal those of a
 * FACTOR_U64 actor of a runtime with the default max_factor_n (2^62 - 1); a
 * runtime created with a smaller limit refuses larger n, which this call
 * still factors.  Work is enqueued on `stream` (cudaStream_t, NULL = the
 * legacy default stream) and the call returns at once; the replies are
 * complete when the stream reaches this point.  The caller owns both arrays.
 *
 * It allocates nothing: the two scratch words per number live in a fixed
 * array of CAF_GPU_FACTOR_STATIC_MAX entries (32 KB) compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  The address is kept for the life of the process, so
 * the device's primary context must not be reset (cudaDeviceReset) after the
 * first call.  All calls share the array, so calls whose work overlaps
 * on the GPU (other streams, other threads) race and must not be issued; each
 * call resets the words it uses before its kernel runs.
 *
 * Errors: CAF_GPU_EINVAL if count > CAF_GPU_FACTOR_STATIC_MAX or a pointer is
 * NULL (nothing is launched); CAF_GPU_ECUDA if the set-up or a launch fails. */
#define CAF_GPU_FACTOR_STATIC_MAX 4096u
int caf_gpu_factor_static(const uint64_t *d_n, uint32_t count, caf_gpu_dreply *d_replies, void *stream);

const char *caf_gpu_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CAF_GPU_H */
