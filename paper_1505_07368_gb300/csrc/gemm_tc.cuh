// GEMM payload: C = A * B for square FP32 matrices (n x n, row-major,
// leading dimension n) on the 5th-generation tensor cores.  This is the
// matrix-multiply actor of Sec. 3.6 (an OpenCL kernel taking two float
// matrices and producing their product), computed as
//
//   BF16:            C = bf16(A) * bf16(B)                     (FP32 accumulate)
//   split-BF16x3:    C = hi(A)*hi(B) + [hi(A)*lo(B) + lo(A)*hi(B)]
//                    with hi(x) = bf16_rn(x), lo(x) = bf16_rn(x - hi(x))
//
// One CTA computes one 128 x 128 output tile.  k runs in slices of 64 (the
// FP32 staging unit) and blocks of 16 (one MMA step, the BF16 unit):
//   * one thread stages each slice with three tensor copies (TMA) described
//     by per-matrix tensor maps: A as two 32-wide k halves with the 128-byte
//     swizzle, B as one 128-column x 64-k box.  The copies zero-fill whatever
//     lies outside the n x n matrices, so the edge tiles need no masking.  Two
//     slices are in flight; the last converter warp done with a stage issues
//     its refill;
//   * each of the 8 converter warps rounds its share of the slice to BF16 (hi,
//     and lo for the split form) into a ring of operand slots, one 16-wide k
//     block per slot, laid out K-major with the 32-byte swizzle the tensor
//     core reads.  Warp w converts 16 rows of A for every block and 8 k rows of
//     B (one half of one block's B^T, transposed on the way);
//   * one thread issues tcgen05.mma per block (M=128, kind::f16, BF16 in, FP32
//     accumulators in tensor memory) and frees the slot with tcgen05.commit.
//     The split form is two MMAs: hi(A) against [hi(B); lo(B)] as one N=256
//     operand (accumulator columns 0..255), then lo(A) against hi(B) into
//     columns 128..255, so the tile is D[0..127] + D[128..255];
//   * the converter warps read the accumulators with tcgen05.ld and store the
//     tile (masked at the matrix edge).
// The slot ring lets conversion of block u overlap the MMAs of earlier
// blocks; the staging ring lets the copies of slice s+2 overlap both.
// Tensor maps need 16-byte aligned rows; when n is not a multiple of 4 (or an
// operand is unaligned, or no maps were built) the converters read global
// memory directly instead.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace cafgpu {

constexpr uint32_t kGemmBM = 128;          // tile rows (MMA M)
constexpr uint32_t kGemmBN = 128;          // tile columns (MMA N of one product)
constexpr uint32_t kGemmBK = 64;           // k per FP32 staging slice
constexpr uint32_t kGemmKB = 16;           // k per BF16 block (one MMA)
constexpr uint32_t kGemmBlocks = kGemmBK / kGemmKB;   // blocks per slice
constexpr uint32_t kGemmConvWarps = 8;
constexpr uint32_t kGemmPlaneBytes = kGemmBM * kGemmKB * 2;   // 4 KB: 128 rows x 16 k BF16
constexpr uint32_t kGemmTmemCols = 256;

// One BF16 operand slot: 128 rows x 16 k per plane, K-major, 32-byte swizzle.
// b_hi and b_lo are adjacent so the split form reads them as one 256-row B.
struct GemmBfSlot {
    uint8_t a_hi[kGemmPlaneBytes];
    uint8_t a_lo[kGemmPlaneBytes];
    uint8_t b_hi[kGemmPlaneBytes];
    uint8_t b_lo[kGemmPlaneBytes];
};
static_assert(sizeof(GemmBfSlot) == kGemmSlotBytes, "slot size");
// One FP32 staging stage: the A slice as two 32-wide k halves (128 rows of
// 128 bytes, 128-byte swizzle: 16-byte chunk q of row r at chunk q ^ (r & 7)),
// and the B slice (64 rows of k, 128 columns, dense).
struct GemmF32Stage {
    float a[2][kGemmBM * 32];
    float b[kGemmBK * kGemmBN];
};
static_assert(sizeof(GemmF32Stage) == kGemmStageBytes, "stage size");
// Operand area of one GEMM CTA (1024-byte aligned).
struct GemmOps {
    GemmBfSlot bf[kGemmBfSlots];
    GemmF32Stage f32[kGemmF32Stages];
};
static_assert(sizeof(GemmOps) == kGemmOpsBytes, "operand area size");
struct GemmSmem {
    GemmOps ops;
    GemmBars bars;
};

// One output tile's operands.  tmap_a / tmap_b: tensor maps of A and B
// (kernel-parameter memory), or null for the direct path.
struct GemmArgs {
    const float *A, *B;
    float *C;
    const void *tmap_a, *tmap_b;
    uint32_t n, tm, tn;
    bool split;
};

// Barrier phases of one CTA across the tiles it computes.
struct GemmCounters {
    uint32_t f32_uses;   // slices staged so far (stage = use % kGemmF32Stages)
    uint32_t bf_uses;    // BF16 blocks converted so far (slot = use % kGemmBfSlots)
    uint32_t tiles;      // tiles finished (done barrier phase)
    uint32_t pk_uses;    // packed k blocks streamed so far (slot = use % kPackSlots)
};

// ---- tensor copies ------------------------------------------------------
// 2-D tiled tensor copy global -> shared (box at element coordinates x
// (innermost) and y), completing on an mbarrier.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int32_t x, int32_t y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ---- tcgen05 wrappers -------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_result, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_result)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, both K-major, kind::f16.
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 32 lanes x 32 columns of 32-bit accumulator: thread t gets row (lane base + t).
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 32-byte swizzle (rows of
// 32 bytes = one 16-wide k block, so one swizzle atom spans the MMA's K and
// the leading byte offset is unused), 8-row groups 256 bytes apart (stride
// byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw32(const void *p) {
    const uint64_t addr = smem_u32(p);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(256 >> 4) << 32) | (1ull << 46) |
           (6ull << 61);
}

// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t gemm_idesc(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Byte offset of the 8-element chunk c (k 8c..8c+7) of row r in a 128-row x
// 16-k K-major plane with the 32-byte swizzle (address bit 4 ^= bit 7).
__device__ __forceinline__ uint32_t sw32_offset(uint32_t r, uint32_t c) {
    return r * 32u + ((c ^ ((r >> 2) & 1u)) << 4);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Round 8 floats to BF16 (hi) and, for the split form, the BF16 of the
// remainders (lo); write each 16-byte result chunk.
__device__ __forceinline__ void convert8(const float (&x)[8], uint8_t *hi_dst, uint8_t *lo_dst, bool split) {
    uint4 h;
    h.x = pack_bf16x2(x[0], x[1]);
    h.y = pack_bf16x2(x[2], x[3]);
    h.z = pack_bf16x2(x[4], x[5]);
    h.w = pack_bf16x2(x[6], x[7]);
    *reinterpret_cast<uint4 *>(hi_dst) = h;
    if (split) {
        const __nv_bfloat162 *hb = reinterpret_cast<const __nv_bfloat162 *>(&h);
        float r[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(hb[i]);
            r[2 * i] = x[2 * i] - f.x;
            r[2 * i + 1] = x[2 * i + 1] - f.y;
        }
        uint4 l;
        l.x = pack_bf16x2(r[0], r[1]);
        l.y = pack_bf16x2(r[2], r[3]);
        l.z = pack_bf16x2(r[4], r[5]);
        l.w = pack_bf16x2(r[6], r[7]);
        *reinterpret_cast<uint4 *>(lo_dst) = l;
    }
}

// Stage slice kb of tile (tm, tn) into S (one thread): A's two k halves and
// B's 64 k rows.  The full box is always written (zero outside the matrix),
// so the transaction count is the stage size.
__device__ __forceinline__ void gemm_stage_issue(const GemmArgs &g, uint32_t kb, GemmF32Stage &S, uint64_t *bar) {
    const int32_t k0 = (int32_t)(kb * kGemmBK), row0 = (int32_t)(g.tm * kGemmBM), col0 = (int32_t)(g.tn * kGemmBN);
    fence_proxy_async_smem();   // earlier generic reads of this stage before the async writes
    mbar_arrive_expect_tx(bar, kGemmStageBytes);
    tma_load_2d(S.a[0], g.tmap_a, k0, row0, bar);
    tma_load_2d(S.a[1], g.tmap_a, k0 + 32, row0, bar);
    tma_load_2d(S.b, g.tmap_b, col0, k0, bar);
}

// B part of slice kb: warp w's 8 k rows (k0+8w..) for all 128 columns, as
// chunk w&1 of block w>>1's B^T rows.  Lane: columns lane + 32i.  Source: the
// staged slice, or global memory (kDirect, masked at the matrix edge).
template <bool kDirect>
__device__ __forceinline__ void gemm_convert_b(const GemmArgs &g, const GemmF32Stage &S, uint32_t k0,
                                               GemmBfSlot &slot, uint32_t w) {
    const uint32_t lane = lane_id();
    const uint32_t c = w & 1u, gk = k0 + 8 * w;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t col = lane + 32u * i, gc = g.tn * kGemmBN + col;
        float x[8];
#pragma unroll
        for (uint32_t j = 0; j < 8; ++j) {
            if (kDirect)
                x[j] = (gc < g.n && gk + j < g.n) ? __ldg(g.B + (size_t)(gk + j) * g.n + gc) : 0.0f;
            else
                x[j] = S.b[(8 * w + j) * kGemmBN + col];
        }
        const uint32_t off = sw32_offset(col, c);
        convert8(x, slot.b_hi + off, slot.b_lo + off, g.split);
    }
}

// A part of block j of slice kb: warp w's rows 16w..16w+15, k 16j..16j+15.
// Lane: row 16w + (lane & 15), chunk lane >> 4.
template <bool kDirect>
__device__ __forceinline__ void gemm_convert_a(const GemmArgs &g, const GemmF32Stage &S, uint32_t k0,
                                               GemmBfSlot &slot, uint32_t w, uint32_t j) {
    const uint32_t lane = lane_id();
    const uint32_t r = 16 * w + (lane & 15u), c = lane >> 4;
    float x[8];
    if (kDirect) {
        const uint32_t gr = g.tm * kGemmBM + r, gk = k0 + 16 * j + 8 * c;
#pragma unroll
        for (uint32_t e = 0; e < 8; ++e)
            x[e] = (gr < g.n && gk + e < g.n) ? __ldg(g.A + (size_t)gr * g.n + gk + e) : 0.0f;
    } else {
        // 16-byte chunks q, q+1 of row r in k half j>>1
        const uint8_t *row = reinterpret_cast<const uint8_t *>(S.a[j >> 1]) + r * 128u;
        const uint32_t q = 4 * (j & 1u) + 2 * c;
        const float4 lo = *reinterpret_cast<const float4 *>(row + ((q ^ (r & 7u)) << 4));
        const float4 hi = *reinterpret_cast<const float4 *>(row + (((q + 1) ^ (r & 7u)) << 4));
        x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
        x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
    }
    const uint32_t off = sw32_offset(r, c);
    convert8(x, slot.a_hi + off, slot.a_lo + off, g.split);
}

}  // namespace cafgpu

namespace cafgpu {

constexpr uint32_t kGemmThreads = (kGemmConvWarps + 1) * 32;   // converters + one MMA warp
constexpr uint32_t kGemmSmemBytes = (uint32_t)sizeof(GemmSmem) + 1024;  // + alignment slack

// 1024-byte aligned GemmSmem inside dynamic shared memory.
__device__ __forceinline__ GemmSmem &gemm_smem(uint8_t *raw) {
    const uint32_t a = smem_u32(raw);
    const uint32_t pad = (1024u - (a & 1023u)) & 1023u;
    return *reinterpret_cast<GemmSmem *>(raw + pad);
}

// Barrier set-up and tensor-memory allocation, run by warp kGemmConvWarps
// (the caller synchronises the CTA afterwards, with tcgen05 fences).
__device__ __forceinline__ void gemm_bars_init(GemmBars &Bb, uint32_t tmem_cols = kGemmTmemCols) {
    if (lane_id() == 0) {
        for (uint32_t s = 0; s < kGemmF32Stages; ++s) {
            mbar_init(&Bb.f32_full[s], 1);
            Bb.f32_read[s] = 0;
        }
        for (uint32_t s = 0; s < kGemmBfSlots; ++s) {
            mbar_init(&Bb.bf_full[s], kGemmConvWarps);
            mbar_init(&Bb.bf_empty[s], 1);
        }
        for (uint32_t s = 0; s < kPackSlots; ++s) {
            mbar_init(&Bb.pk_full[s], 1);
            mbar_init(&Bb.pk_empty[s], 1);
        }
        for (uint32_t b = 0; b < 2; ++b) {
            mbar_init(&Bb.acc_full[b], 1);
            mbar_init(&Bb.acc_empty[b], 4);
        }
        mbar_init(&Bb.done, 1);
        fence_barrier_init();
    }
    __syncwarp();
    tmem_alloc(&Bb.tmem, tmem_cols);
}

__device__ __forceinline__ void gemm_cta_init(GemmSmem &S) {
    if ((threadIdx.x >> 5) == kGemmConvWarps) gemm_bars_init(S.bars);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void gemm_cta_exit(GemmSmem &S) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == kGemmConvWarps) {
        tc_fence_after();
        tmem_dealloc(S.bars.tmem, kGemmTmemCols);
    }
}

// Bounded mbarrier wait; false after `limit_ns` (the caller records the error).
__device__ __forceinline__ bool gemm_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    WaitClock wc(limit_ns);
    while (!mbar_try_wait(bar, parity)) {
        if (!wc.again()) return false;
    }
    return true;
}

// Whole-CTA synchronisation for gemm_tile.
struct CtaSyncAll {
    __device__ __forceinline__ void operator()() const {
        __syncwarp();   // the MMA warp's lane 0 diverged while issuing
        __syncthreads();
    }
};

// Wait (warp-wide) until slot use u may be overwritten: the MMAs of use
// u - kGemmBfSlots have completed.
__device__ __forceinline__ bool gemm_slot_free(GemmBars &Bb, uint32_t u, uint64_t limit_ns) {
    if (u < kGemmBfSlots) return true;
    return gemm_wait(&Bb.bf_empty[u % kGemmBfSlots], (u / kGemmBfSlots - 1u) & 1u, limit_ns);
}

// One slice of converter warp w: its B part, then the A parts of all the
// slice's blocks (independent work the warp can overlap), then one publish of
// every block to the MMA thread.  Returns false if a wait expired.
template <bool kDirect>
__device__ __forceinline__ bool gemm_convert_slice(const GemmArgs &g, const GemmF32Stage &S, uint32_t k0,
                                                   GemmOps &O, GemmBars &Bb, uint32_t u0, uint32_t w,
                                                   uint64_t limit_ns) {
    const uint32_t lane = lane_id();
    const uint32_t jb = w >> 1, ub = u0 + jb;
    bool ok = true;
#pragma unroll
    for (uint32_t j = 0; j < kGemmBlocks; ++j) ok = ok && gemm_slot_free(Bb, u0 + j, limit_ns);
    if (!__all_sync(0xFFFFFFFFu, ok)) return false;
    gemm_convert_b<kDirect>(g, S, k0, O.bf[ub % kGemmBfSlots], w);
#pragma unroll
    for (uint32_t j = 0; j < kGemmBlocks; ++j)
        gemm_convert_a<kDirect>(g, S, k0, O.bf[(u0 + j) % kGemmBfSlots], w, j);
    fence_proxy_async_smem();   // generic-proxy writes -> tensor-core (async proxy) reads
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (uint32_t j = 0; j < kGemmBlocks; ++j)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                             smem_u32(&Bb.bf_full[(u0 + j) % kGemmBfSlots]))
                         : "memory");
    }
    return true;
}

// Epilogue of a tile, converter warps 0..7: wait for the last MMA (done
// barrier, phase `tiles`), read the accumulators (warp w: TMEM lanes
// 32*(w%4).., columns 64*(w/4)..; the split form adds columns 128.. to them)
// and store the tile of C, masked at the matrix edge.  Returns false if the
// wait expired or `ok` was already false.
__device__ __forceinline__ bool gemm_epilogue(float *__restrict__ C, uint32_t n, uint32_t tm, uint32_t tn,
                                              bool split, GemmBars &Bb, uint32_t tiles, bool ok,
                                              uint64_t limit_ns) {
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    bool dok = ok && gemm_wait(&Bb.done, tiles & 1u, limit_ns);
    dok = __all_sync(0xFFFFFFFFu, dok);
    if (!dok) return false;
    tc_fence_after();
    const uint32_t row0 = (warp & 3u) * 32u, col0 = (warp >> 2) * 64u;
    const uint32_t gr = tm * kGemmBM + row0 + lane;
#pragma unroll
    for (uint32_t cc = 0; cc < 64; cc += 32) {
        uint32_t r[32];
        tmem_ld_32x32(Bb.tmem + (row0 << 16) + col0 + cc, r);
        if (split) {
            uint32_t r2[32];
            tmem_ld_32x32(Bb.tmem + (row0 << 16) + kGemmBN + col0 + cc, r2);
#pragma unroll
            for (uint32_t j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(r2[j]));
        }
        if (gr < n) {
            float *crow = C + (size_t)gr * n;
            const uint32_t gc0 = tn * kGemmBN + col0 + cc;
            if (gc0 + 32 <= n && (reinterpret_cast<uintptr_t>(crow + gc0) & 15u) == 0) {
#pragma unroll
                for (uint32_t j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4 *>(crow + gc0 + j) =
                        make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                    __uint_as_float(r[j + 3]));
            } else {
#pragma unroll
                for (uint32_t j = 0; j < 32; ++j)
                    if (gc0 + j < n) crow[gc0 + j] = __uint_as_float(r[j]);
            }
        }
    }
    return true;
}

// Issue the MMAs of one 16-wide k block held in `sl` (one thread).  BF16:
// hi(A) hi(B)^T, N = 128.  Split: hi(A) [hi(B); lo(B)]^T as one N = 256
// product (columns 0..255), then lo(A) hi(B)^T into columns 128..255.
// `first`: the tile's first block (overwrite instead of accumulate).
// a_hi, a_lo, b_hi: the block's planes; b_lo must follow b_hi directly.
__device__ __forceinline__ void gemm_mma_planes(const void *a_hi, const void *a_lo, const void *b_hi, uint32_t tmem,
                                                bool split, bool first) {
    const uint32_t id128 = gemm_idesc(kGemmBM, kGemmBN), id256 = gemm_idesc(kGemmBM, 2 * kGemmBN);
    const uint64_t ah = smem_desc_sw32(a_hi), bh = smem_desc_sw32(b_hi);
    if (split) {
        tc_mma_f16(tmem, ah, bh, id256, first ? 0u : 1u);
        tc_mma_f16(tmem + kGemmBN, smem_desc_sw32(a_lo), bh, id128, 1u);
    } else {
        tc_mma_f16(tmem, ah, bh, id128, first ? 0u : 1u);
    }
}
__device__ __forceinline__ void gemm_mma_block(GemmBfSlot &sl, uint32_t tmem, bool split, bool first) {
    gemm_mma_planes(sl.a_hi, sl.a_lo, sl.b_hi, tmem, split, first);
}

// Compute one output tile of C = A * B with the whole CTA (converter warps
// 0..7 and the MMA warp kGemmConvWarps).  `K` carries the barrier phases
// across the tiles this CTA computes.  Returns false if a bounded wait
// expired.
template <class CtaSync>
__device__ bool gemm_tile(const GemmArgs &g, GemmOps &O, GemmBars &Bb, GemmCounters &K, uint64_t limit_ns,
                          CtaSync cta_sync) {
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t n = g.n, nk = (n + kGemmBK - 1) / kGemmBK;
    const bool staged = g.tmap_a != nullptr;
    bool ok = true;
    if (warp < kGemmConvWarps) {
        const uint32_t w = warp;
        if (staged && lane == 0) {
            if (w == 0)
                for (uint32_t kb = 0; kb < kGemmF32Stages && kb < nk; ++kb) {
                    const uint32_t st = (K.f32_uses + kb) % kGemmF32Stages;
                    gemm_stage_issue(g, kb, O.f32[st], &Bb.f32_full[st]);
                }
        }
        __syncwarp();
        uint32_t kb = 0;
#pragma unroll 1
        for (; kb < nk; ++kb) {
            const uint32_t u0 = K.bf_uses + kb * kGemmBlocks;
            if (!staged) {
                ok = gemm_convert_slice<true>(g, O.f32[0], kb * kGemmBK, O, Bb, u0, w, limit_ns);
            } else {
                const uint32_t fu = K.f32_uses + kb, st = fu % kGemmF32Stages;
                bool okw = gemm_wait(&Bb.f32_full[st], (fu / kGemmF32Stages) & 1u, limit_ns);
                if (!__all_sync(0xFFFFFFFFu, okw)) { ok = false; break; }
                ok = gemm_convert_slice<false>(g, O.f32[st], kb * kGemmBK, O, Bb, u0, w, limit_ns);
                // release the stage; the last warp out issues its refill
                if (ok && lane == 0) {
                    __threadfence_block();
                    const uint32_t prev = atomicAdd(&Bb.f32_read[st], 1u);
                    if ((prev + 1) % kGemmConvWarps == 0 && kb + kGemmF32Stages < nk)
                        gemm_stage_issue(g, kb + kGemmF32Stages, O.f32[st], &Bb.f32_full[st]);
                }
                __syncwarp();
            }
            if (!ok) break;
        }
        // after an expired wait, let copies possibly still in flight land
        // (bounded) before the shared memory can be reused
        for (uint32_t q = kb; staged && !ok && q < nk && q < kb + kGemmF32Stages; ++q) {
            const uint32_t fu = K.f32_uses + q;
            gemm_wait(&Bb.f32_full[fu % kGemmF32Stages], (fu / kGemmF32Stages) & 1u, limit_ns);
        }
    } else if (lane == 0) {
        const uint32_t nb = nk * kGemmBlocks;
        for (uint32_t i = 0; i < nb && ok; ++i) {
            const uint32_t u = K.bf_uses + i, s = u % kGemmBfSlots;
            ok = gemm_wait(&Bb.bf_full[s], (u / kGemmBfSlots) & 1u, limit_ns);
            if (!ok) break;
            tc_fence_after();
            gemm_mma_block(O.bf[s], Bb.tmem, g.split, i == 0);
            tc_commit(&Bb.bf_empty[s]);
        }
        tc_commit(&Bb.done);
    }
    if (warp == kGemmConvWarps) __syncwarp();
    K.f32_uses += staged ? nk : 0;
    K.bf_uses += nk * kGemmBlocks;
    if (warp < kGemmConvWarps) ok = gemm_epilogue(g.C, n, g.tm, g.tn, g.split, Bb, K.tiles, ok, limit_ns);
    ++K.tiles;
    // the next tile's MMAs overwrite the accumulators: every epilogue read
    // must be complete first
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    return ok;
}

}  // namespace cafgpu
