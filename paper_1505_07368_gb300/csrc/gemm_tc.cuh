// GEMM payload: C = A * B for square FP32 matrices (n x n, row-major,
// leading dimension n) on the 5th-generation tensor cores.  This is the
// matrix-multiply actor of Sec. 3.6 (an OpenCL kernel taking two float
// matrices and producing their product), computed as
//
//   BF16:            C = bf16(A) * bf16(B)                     (FP32 accumulate)
//   split-BF16x3:    C = hi(A)*hi(B) + hi(A)*lo(B) + lo(A)*hi(B)
//                    with hi(x) = bf16_rn(x), lo(x) = bf16_rn(x - hi(x))
//
// One CTA computes one 128 x 128 output tile:
//   * 8 converter warps load FP32 operand blocks (128 rows x 64 k) from
//     global memory, round them to BF16 (hi, and lo for the split form) and
//     store them into shared memory in the canonical K-major 128-byte-swizzle
//     layout the tensor core reads (B is transposed on the way, so both
//     operands are K-major);
//   * one thread issues tcgen05.mma (M=128, N=128, K=16, kind::f16, BF16 in,
//     FP32 accumulator in tensor memory) and commits each stage back to the
//     converters through an mbarrier;
//   * the same 8 warps then read the accumulator with tcgen05.ld and store
//     the tile (masked at the matrix edge).
// Two operand stages let the conversion of block k+1 overlap the MMAs of
// block k.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace cafgpu {

constexpr uint32_t kGemmBM = 128;          // tile rows (MMA M)
constexpr uint32_t kGemmBN = 128;          // tile columns (MMA N)
constexpr uint32_t kGemmBK = 64;           // k per stage: one 128-byte swizzle atom of BF16
constexpr uint32_t kGemmStages = 2;
constexpr uint32_t kGemmConvWarps = 8;
constexpr uint32_t kGemmOperandBytes = kGemmBM * kGemmBK * 2;   // 16 KB per operand tile
constexpr uint32_t kGemmTmemCols = 128;

// Operand tiles of one GEMM CTA (1024-byte aligned: the swizzle pattern
// repeats every 1024 bytes).
struct GemmOps {
    uint8_t a_hi[kGemmStages][kGemmOperandBytes];
    uint8_t b_hi[kGemmStages][kGemmOperandBytes];
    uint8_t a_lo[kGemmStages][kGemmOperandBytes];
    uint8_t b_lo[kGemmStages][kGemmOperandBytes];
};
static_assert(sizeof(GemmOps) == kGemmOpsBytes, "operand area size");
static_assert(kGemmStages == 2, "GemmBars holds two stages");
struct GemmSmem {
    GemmOps ops;
    GemmBars bars;
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

// Converter thread work for one k block: this CTA's 256 converter threads
// write A (rows tm*128.., k kb*64..) and B^T (rows = columns tn*128.. of B).
// Each thread produces 4 chunks of A and 4 of B (one chunk = 8 consecutive k).
__device__ __forceinline__ void gemm_convert_block(const float *__restrict__ A, const float *__restrict__ B,
                                                   uint32_t n, uint32_t tm, uint32_t tn, uint32_t kb,
                                                   uint8_t *a_hi, uint8_t *b_hi, uint8_t *a_lo, uint8_t *b_lo,
                                                   bool split, uint32_t tid) {
    const uint32_t k0 = kb * kGemmBK;
    // A: chunk id c in [0, 1024): row = c / 8, kchunk = c % 8; thread handles c = tid + 256 i
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t c = tid + 256u * i;
        const uint32_t r = c >> 3, kc = c & 7u;
        const uint32_t gr = tm * kGemmBM + r, gk = k0 + kc * 8;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (gr < n && gk + j < n) ? __ldg(A + (size_t)gr * n + gk + j) : 0.0f;
        const uint32_t off = sw128_offset(r, kc);
        convert8(x, a_hi + off, a_lo + off, split);
    }
    // B^T: row = column of B (col), k chunk; thread layout: lanes over columns
    // so that each k row of B is read contiguously by a warp.
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t c = tid + 256u * i;
        const uint32_t col = c & 127u, kc = c >> 7;
        const uint32_t gc = tn * kGemmBN + col, gk = k0 + kc * 8;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (gc < n && gk + j < n) ? __ldg(B + (size_t)(gk + j) * n + gc) : 0.0f;
        const uint32_t off = sw128_offset(col, kc);
        convert8(x, b_hi + off, b_lo + off, split);
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
        for (uint32_t s = 0; s < kGemmStages; ++s) {
            mbar_init(&Bb.full[s], kGemmConvWarps);
            mbar_init(&Bb.empty[s], 1);
        }
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

// Compute output tile (tm, tn) of C = A * B with the whole CTA.
// `stage_uses` counts operand-stage uses over the CTA's life and `tiles`
// the tiles it has computed (barrier phases follow from both).  Returns false
// if a bounded wait expired.
// Whole-CTA synchronisation for gemm_tile.
struct CtaSyncAll {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// `cta_sync` synchronises the warps taking part (all kGemmConvWarps + 1).
template <class CtaSync>
__device__ bool gemm_tile(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C,
                          uint32_t n, uint32_t tm, uint32_t tn, bool split, GemmOps &S, GemmBars &Bb,
                          uint32_t &stage_uses, uint32_t &tiles, uint64_t limit_ns, CtaSync cta_sync) {
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t nk = (n + kGemmBK - 1) / kGemmBK;
    bool ok = true;
    if (warp < kGemmConvWarps) {
        for (uint32_t kb = 0; kb < nk && ok; ++kb) {
            const uint32_t it = stage_uses + kb;
            const uint32_t st = it % kGemmStages, use = it / kGemmStages;
            if (use >= 1) ok = gemm_wait(&Bb.empty[st], (use - 1) & 1u, limit_ns);
            if (!__all_sync(0xFFFFFFFFu, ok)) { ok = false; break; }
            gemm_convert_block(A, B, n, tm, tn, kb, S.a_hi[st], S.b_hi[st], S.a_lo[st], S.b_lo[st], split,
                               threadIdx.x);
            fence_proxy_async_smem();   // generic-proxy writes -> tensor-core (async proxy) reads
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&Bb.full[st])) : "memory");
        }
    } else if (lane == 0) {
        const uint32_t idesc = gemm_idesc(kGemmBM, kGemmBN);
        for (uint32_t kb = 0; kb < nk && ok; ++kb) {
            const uint32_t it = stage_uses + kb;
            const uint32_t st = it % kGemmStages, use = it / kGemmStages;
            ok = gemm_wait(&Bb.full[st], use & 1u, limit_ns);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ah = smem_desc_sw128(S.a_hi[st]), bh = smem_desc_sw128(S.b_hi[st]);
            const uint64_t al = smem_desc_sw128(S.a_lo[st]), bl = smem_desc_sw128(S.b_lo[st]);
#pragma unroll
            for (uint32_t k16 = 0; k16 < kGemmBK / 16; ++k16) {
                const uint64_t ko = (k16 * 32u) >> 4;   // 16 BF16 = 32 bytes along k inside the swizzle atom
                tc_mma_f16(Bb.tmem, ah + ko, bh + ko, idesc, (kb | k16) != 0);
                if (split) {
                    tc_mma_f16(Bb.tmem, ah + ko, bl + ko, idesc, 1u);
                    tc_mma_f16(Bb.tmem, al + ko, bh + ko, idesc, 1u);
                }
            }
            tc_commit(&Bb.empty[st]);
        }
        tc_commit(&Bb.done);
    }
    stage_uses += nk;
    // epilogue: converter warps read the accumulator (warp w: TMEM lanes
    // 32*(w%4).., columns 64*(w/4)..) and store the tile
    if (warp < kGemmConvWarps) {
        bool dok = ok && gemm_wait(&Bb.done, tiles & 1u, limit_ns);
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
#pragma unroll
                    for (uint32_t j = 0; j < 32; ++j)
                        if (gc0 + j < n) crow[gc0 + j] = __uint_as_float(r[j]);
                }
            }
        }
        ok = ok && dok;
    }
    ++tiles;
    // the next tile's MMAs overwrite the accumulator: every epilogue read
    // must be complete first
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    return ok;
}

}  // namespace cafgpu
