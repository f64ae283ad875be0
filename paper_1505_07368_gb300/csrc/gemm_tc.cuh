// GEMM payload: C = A * B for square FP32 matrices (n x n, row-major,
// leading dimension n) on the 5th-generation tensor cores.  This is the
// matrix-multiply actor of Sec. 3.6 (an OpenCL kernel taking two float
// matrices and producing their product), computed as
//
//   BF16:            C = bf16(A) * bf16(B)                     (FP32 accumulate)
//   split-BF16x3:    C = hi(A)*hi(B) + hi(A)*lo(B) + lo(A)*hi(B)
//                    with hi(x) = bf16_rn(x), lo(x) = bf16_rn(x - hi(x))
//
// One CTA computes one 128 x 128 output tile, k in blocks of 64:
//   * each of the 8 converter warps owns a slice of every k block -- 16 rows
//     of the A block and 8 rows (k) of the B block -- and stages it into
//     shared memory with bulk asynchronous copies (one per row, completing on
//     the warp's own mbarrier), two blocks ahead;
//   * the warp then rounds its FP32 slice to BF16 (hi, and lo for the split
//     form) and writes it in the canonical K-major 128-byte-swizzle layout
//     the tensor core reads (B transposed on the way, so both operands are
//     K-major), and refills the staging stage with the block two ahead;
//   * one thread issues tcgen05.mma (M=128, N=128, K=16, kind::f16, BF16 in,
//     FP32 accumulator in tensor memory) and commits the operand buffer back
//     to the converters through an mbarrier;
//   * the converter warps read the accumulator with tcgen05.ld and store the
//     tile (masked at the matrix edge).
// Bulk copies need 16-byte aligned rows; when n is not a multiple of 4 (or an
// operand is unaligned) the converters read global memory directly instead.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace cafgpu {

constexpr uint32_t kGemmBM = 128;          // tile rows (MMA M)
constexpr uint32_t kGemmBN = 128;          // tile columns (MMA N)
constexpr uint32_t kGemmBK = 64;           // k per stage: one 128-byte swizzle atom of BF16
constexpr uint32_t kGemmConvWarps = 8;
constexpr uint32_t kGemmOperandBytes = kGemmBM * kGemmBK * 2;   // 16 KB per BF16 operand tile
constexpr uint32_t kGemmTmemCols = 128;

// Operand tiles of one GEMM CTA (1024-byte aligned: the swizzle pattern
// repeats every 1024 bytes), then the FP32 staging.
struct GemmOps {
    uint8_t a_hi[kGemmOperandBytes];
    uint8_t b_hi[kGemmOperandBytes];
    uint8_t a_lo[kGemmOperandBytes];
    uint8_t b_lo[kGemmOperandBytes];
    float a32[2][kGemmBM * kGemmBK];   // A block: 128 rows x 64 k
    float b32[2][kGemmBK * kGemmBN];   // B block: 64 rows (k) x 128 columns
};
static_assert(sizeof(GemmOps) == kGemmOpsBytes, "operand area size");
struct GemmSmem {
    GemmOps ops;
    GemmBars bars;
};

// Barrier phases of one CTA across the tiles it computes.
struct GemmCounters {
    uint32_t f32_uses;   // k blocks staged so far (staging stage = use & 1)
    uint32_t bf_uses;    // k blocks converted so far (one BF16 operand buffer)
    uint32_t tiles;      // tiles finished (done barrier phase)
};

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

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p) {
    const uint64_t addr = smem_u32(p);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t gemm_idesc(uint32_t m, uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

// Byte offset of element (row r, k) in a 128-row x 64-k K-major SW128 tile.
__device__ __forceinline__ uint32_t sw128_offset(uint32_t r, uint32_t chunk /* k / 8 */) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + (((chunk ^ r) & 7u) << 4);
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

// Issue the bulk copies of this warp's slice of k block kb into staging
// stage st (warp-collective): A rows 16w..16w+15 of the tile, B rows
// k0+8w..k0+8w+7.  Rows past n are not copied (the converter zero-fills).
__device__ __forceinline__ void gemm_stage_issue(const float *A, const float *B, uint32_t n, uint32_t tm,
                                                 uint32_t tn, uint32_t kb, float *a32, float *b32, uint64_t *bar,
                                                 uint32_t w) {
    const uint32_t lane = lane_id();
    const uint32_t k0 = kb * kGemmBK, col0 = tn * kGemmBN, row0 = tm * kGemmBM + 16 * w;
    const uint32_t a_bytes = min(kGemmBK, n - k0) * 4u;
    const uint32_t b_bytes = min(kGemmBN, n - col0) * 4u;
    const uint32_t na = row0 < n ? min(16u, n - row0) : 0u;
    const uint32_t nb = (k0 + 8 * w) < n ? min(8u, n - (k0 + 8 * w)) : 0u;
    fence_proxy_async_smem();   // earlier generic reads of this stage before the async writes
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(bar, na * a_bytes + nb * b_bytes);
    __syncwarp();
    if (lane < na)
        bulk_g2s(a32 + (16 * w + lane) * kGemmBK, A + (size_t)(row0 + lane) * n + k0, a_bytes, bar);
    else if (lane >= 16 && lane - 16 < nb)
        bulk_g2s(b32 + (8 * w + lane - 16) * kGemmBN, B + (size_t)(k0 + 8 * w + lane - 16) * n + col0, b_bytes,
                 bar);
}

// Convert this warp's slice of k block kb to BF16 (hi, lo) into the operand
// tiles.  Source: the staged FP32 slice, or global memory when `direct`.
__device__ __forceinline__ void gemm_convert_slice(const float *__restrict__ A, const float *__restrict__ B,
                                                   uint32_t n, uint32_t tm, uint32_t tn, uint32_t kb,
                                                   const float *a32, const float *b32, bool direct,
                                                   GemmOps &O, bool split, uint32_t w) {
    const uint32_t lane = lane_id();
    const uint32_t k0 = kb * kGemmBK;
    // A: rows 16w + (c >> 3), k chunk c & 7, for c = lane + 32 i
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t c = lane + 32u * i;
        const uint32_t r = 16 * w + (c >> 3), kc = c & 7u;
        const uint32_t gr = tm * kGemmBM + r, gk = k0 + kc * 8;
        float x[8];
        if (direct) {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = (gr < n && gk + j < n) ? __ldg(A + (size_t)gr * n + gk + j) : 0.0f;
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(a32 + r * kGemmBK + kc * 8);
            const float4 lo = src[0], hi = src[1];
            const float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = (gr < n && gk + j < n) ? v[j] : 0.0f;
        }
        const uint32_t off = sw128_offset(r, kc);
        convert8(x, O.a_hi + off, O.a_lo + off, split);
    }
    // B^T: columns lane + 32 i of the tile, k chunk w (B rows k0+8w .. k0+8w+7)
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t col = lane + 32u * i;
        const uint32_t gc = tn * kGemmBN + col, gk = k0 + 8 * w;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool in = gc < n && gk + j < n;
            x[j] = !in ? 0.0f : (direct ? __ldg(B + (size_t)(gk + j) * n + gc) : b32[(8 * w + j) * kGemmBN + col]);
        }
        const uint32_t off = sw128_offset(col, w);
        convert8(x, O.b_hi + off, O.b_lo + off, split);
    }
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
__device__ __forceinline__ void gemm_bars_init(GemmBars &Bb) {
    if (lane_id() == 0) {
        for (uint32_t s = 0; s < 2; ++s)
            for (uint32_t w = 0; w < kGemmConvWarps; ++w) mbar_init(&Bb.f32_full[s][w], 1);
        mbar_init(&Bb.full, kGemmConvWarps);
        mbar_init(&Bb.empty, 1);
        mbar_init(&Bb.done, 1);
        fence_barrier_init();
    }
    __syncwarp();
    tmem_alloc(&Bb.tmem, kGemmTmemCols);
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

// Compute output tile (tm, tn) of C = A * B with the whole CTA (converter
// warps 0..7 and the MMA warp kGemmConvWarps).  `K` carries the barrier
// phases across the tiles this CTA computes.  Returns false if a bounded wait
// expired.
template <class CtaSync>
__device__ bool gemm_tile(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C,
                          uint32_t n, uint32_t tm, uint32_t tn, bool split, GemmOps &O, GemmBars &Bb,
                          GemmCounters &K, uint64_t limit_ns, CtaSync cta_sync) {
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t nk = (n + kGemmBK - 1) / kGemmBK;
    // bulk copies need 16-byte aligned rows
    const bool direct = (n & 3u) != 0 || (reinterpret_cast<uintptr_t>(A) & 15u) != 0 ||
                        (reinterpret_cast<uintptr_t>(B) & 15u) != 0;
    bool ok = true;
    if (warp < kGemmConvWarps) {
        const uint32_t w = warp;
        if (!direct) {
            for (uint32_t kb = 0; kb < 2 && kb < nk; ++kb) {
                const uint32_t st = (K.f32_uses + kb) & 1u;
                gemm_stage_issue(A, B, n, tm, tn, kb, O.a32[st], O.b32[st], &Bb.f32_full[st][w], w);
            }
        }
        for (uint32_t kb = 0; kb < nk; ++kb) {
            const uint32_t fu = K.f32_uses + kb, bu = K.bf_uses + kb;
            const uint32_t st = fu & 1u;
            bool okw = true;
            if (!direct) okw = gemm_wait(&Bb.f32_full[st][w], (fu >> 1) & 1u, limit_ns);
            if (okw && bu >= 1) okw = gemm_wait(&Bb.empty, (bu - 1) & 1u, limit_ns);
            if (!__all_sync(0xFFFFFFFFu, okw)) { ok = false; break; }
            gemm_convert_slice(A, B, n, tm, tn, kb, O.a32[st], O.b32[st], direct, O, split, w);
            fence_proxy_async_smem();   // generic-proxy writes -> tensor-core (async proxy) reads
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&Bb.full)) : "memory");
            if (!direct && kb + 2 < nk)
                gemm_stage_issue(A, B, n, tm, tn, kb + 2, O.a32[st], O.b32[st], &Bb.f32_full[st][w], w);
        }
    } else if (lane == 0) {
        const uint32_t idesc = gemm_idesc(kGemmBM, kGemmBN);
        const uint64_t ah = smem_desc_sw128(O.a_hi), bh = smem_desc_sw128(O.b_hi);
        const uint64_t al = smem_desc_sw128(O.a_lo), bl = smem_desc_sw128(O.b_lo);
        for (uint32_t kb = 0; kb < nk && ok; ++kb) {
            ok = gemm_wait(&Bb.full, (K.bf_uses + kb) & 1u, limit_ns);
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (uint32_t k16 = 0; k16 < kGemmBK / 16; ++k16) {
                const uint64_t ko = (k16 * 32u) >> 4;   // 16 BF16 = 32 bytes along k inside the swizzle atom
                tc_mma_f16(Bb.tmem, ah + ko, bh + ko, idesc, (kb | k16) != 0);
                if (split) {
                    tc_mma_f16(Bb.tmem, ah + ko, bl + ko, idesc, 1u);
                    tc_mma_f16(Bb.tmem, al + ko, bh + ko, idesc, 1u);
                }
            }
            tc_commit(&Bb.empty);
        }
        tc_commit(&Bb.done);
    }
    if (warp == kGemmConvWarps) __syncwarp();
    K.f32_uses += direct ? 0 : nk;
    K.bf_uses += nk;
    // epilogue: converter warps read the accumulator (warp w: TMEM lanes
    // 32*(w%4).., columns 64*(w/4)..) and store the tile
    if (warp < kGemmConvWarps) {
        bool dok = ok && gemm_wait(&Bb.done, K.tiles & 1u, limit_ns);
        dok = __all_sync(0xFFFFFFFFu, dok);
        if (dok) {
            tc_fence_after();
            const uint32_t row0 = (warp & 3u) * 32u, col0 = (warp >> 2) * 64u;
            const uint32_t gr = tm * kGemmBM + row0 + lane;
#pragma unroll
            for (uint32_t cc = 0; cc < 64; cc += 32) {
                uint32_t r[32];
                tmem_ld_32x32(Bb.tmem + (row0 << 16) + col0 + cc, r);
                if (gr < n) {
                    float *crow = C + (size_t)gr * n;
                    const uint32_t gc0 = tn * kGemmBN + col0 + cc;
                    if (gc0 + 32 <= n && (reinterpret_cast<uintptr_t>(crow + gc0) & 15u) == 0) {
#pragma unroll
                        for (uint32_t j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4 *>(crow + gc0 + j) =
                                make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                            __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                    } else {
#pragma unroll
                        for (uint32_t j = 0; j < 32; ++j)
                            if (gc0 + j < n) crow[gc0 + j] = __uint_as_float(r[j]);
                    }
                }
            }
        }
        ok = ok && dok;
    }
    ++K.tiles;
    // the next tile's MMAs overwrite the accumulator: every epilogue read
    // must be complete first
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    return ok;
}

}  // namespace cafgpu
