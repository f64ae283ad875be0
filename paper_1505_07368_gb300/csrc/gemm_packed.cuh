// GEMM payload, packed form (the persistent drain's engine).
//
// The per-message engine (gemm_tc.cuh) rounds FP32 operands to BF16 inside
// every output tile, so a 128-row panel of A is converted once per tile of
// its row, t times for an n x n product with t = ceil(n / 128).  Here each
// GEMM message first has its operands packed, once, by "pack" work items:
//
//   * a pack item converts one 128-row panel of A, or one 128-column panel
//     of B (as rows of B^T), over all k, to BF16 hi (and lo = bf16(x - hi)
//     for the split form), written in exactly the shared-memory image the
//     tensor core reads: per 16-wide k block, a 128-row x 32-byte K-major
//     plane with the 32-byte swizzle (4 KB), hi then lo.  Rows, columns and k
//     past n are written as zeros, so any n works and tiles need no masks;
//   * the CTA that finishes a message's last pack item queues its output
//     tiles (no CTA ever waits for another);
//   * a tile is then a TMA -> tensor-core loop: one thread streams the
//     (panel, block) images of A and B^T into a ring of operand slots with
//     bulk copies (cp.async.bulk), four k blocks per slot and two copies per
//     slot (the blocks of a panel are contiguous), one thread issues
//     tcgen05.mma per block (the same instructions as gemm_tc.cuh), and the
//     converter warps only run the epilogue.  Waits and commits are per
//     slot: an mbarrier wait costs hundreds of cycles even when the phase has
//     completed, more than the MMAs of one block.
//
// Packed size per message: 2 t ceil(n/16) blocks of 4 KB (BF16) or 8 KB
// (split), e.g. 8 MB for a split n = 1024 product.
#pragma once

#include "gemm_tc.cuh"

namespace cafgpu {

constexpr uint32_t kPackPlane = kGemmPlaneBytes;       // 4 KB: 128 rows x 16 k BF16
constexpr uint32_t kPackItemFlag = 0x8000u;            // work item: pack (else tile)

// Operand slots of a packed tile (the drain's GEMM shared-memory area): each
// holds bps consecutive k blocks, the A panel's images first (block b at
// b * blk), then B^T's (at bps * blk).  A block image is its hi plane and,
// for the split form, its lo plane.  bps fills the 64 KB slot for the tile's
// form (kSlotBlocks*): 4 blocks of A and B hi + lo for the split form, 8 of A
// and B for a narrow BF16 tile, 5 of A and two B panels for a wide one.
constexpr uint32_t kPackSlotBytes = 2 * kPackSlotBlocks * 2 * kGemmPlaneBytes;   // 64 KB
struct PackedSlots {
    uint8_t s[kPackSlots][kPackSlotBytes];
};
constexpr uint32_t kSlotBlocksSplit = 4, kSlotBlocksNarrow = 8, kSlotBlocksWide = 5;
static_assert(sizeof(PackedSlots) <= kGemmOpsBytes, "packed slots fit the GEMM area");
static_assert(kSlotBlocksSplit * 2 * 2 * kPackPlane <= kPackSlotBytes, "a split slot fits");
static_assert(kSlotBlocksNarrow * 2 * kPackPlane <= kPackSlotBytes, "a narrow BF16 slot fits");
static_assert(kSlotBlocksWide * 3 * kPackPlane <= kPackSlotBytes, "a wide BF16 slot (A + two B planes) fits");

// Where a message's packed operands live.
struct PackGeom {
    uint8_t *a;      // A panels: block (panel p, k block kb) at a + (p * nkb + kb) * blk
    uint8_t *b;      // B^T panels, same indexing
    uint32_t n, t, nkb, blk;
};

__device__ __forceinline__ PackGeom pack_geom(uint8_t *base, uint32_t n, bool split) {
    PackGeom g;
    g.n = n;
    g.t = (n + kGemmBM - 1) / kGemmBM;
    g.nkb = (n + kGemmKB - 1) / kGemmKB;
    g.blk = split ? 2 * kPackPlane : kPackPlane;
    g.a = base;
    g.b = base + (size_t)g.t * g.nkb * g.blk;
    return g;
}

// Bytes a message of size n needs (host and device).
__host__ __device__ constexpr uint64_t pack_bytes(uint32_t n, bool split) {
    return 2ull * ((n + kGemmBM - 1) / kGemmBM) * ((n + kGemmKB - 1) / kGemmKB) * (split ? 2u : 1u) * kPackPlane;
}

// Pack panel p of A (rows 128p..128p+127), converter warps 0..7.  Warp w
// owns rows 16w..16w+15; lane: row 16w + (lane & 15), 8-wide k chunk
// lane >> 4 of each block.  Eight blocks per step keep eight 32-byte loads
// per lane in flight.
__device__ __forceinline__ void gemm_pack_a(const float *__restrict__ A, const PackGeom &g, uint32_t p,
                                            bool split) {
    const uint32_t w = threadIdx.x >> 5, lane = lane_id();
    const uint32_t r = 16 * w + (lane & 15u), c = lane >> 4, gr = p * kGemmBM + r, n = g.n;
    const bool vec = (n & 3u) == 0 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0;
    const float *row = A + (size_t)min(gr, n - 1) * n;
    const uint32_t off = sw32_offset(r, c);
    uint8_t *dst0 = g.a + (size_t)p * g.nkb * g.blk;
    for (uint32_t kb0 = 0; kb0 < g.nkb; kb0 += 8) {
        float x[8][8];
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) {
            const uint32_t gk = (kb0 + q) * kGemmKB + 8 * c;
            if (vec && gr < n && gk + 8 <= n) {
                const float4 lo = __ldg(reinterpret_cast<const float4 *>(row + gk));
                const float4 hi = __ldg(reinterpret_cast<const float4 *>(row + gk + 4));
                x[q][0] = lo.x; x[q][1] = lo.y; x[q][2] = lo.z; x[q][3] = lo.w;
                x[q][4] = hi.x; x[q][5] = hi.y; x[q][6] = hi.z; x[q][7] = hi.w;
            } else {
#pragma unroll
                for (uint32_t e = 0; e < 8; ++e) x[q][e] = (gr < n && gk + e < n) ? __ldg(row + gk + e) : 0.0f;
            }
        }
#pragma unroll
        for (uint32_t q = 0; q < 8; ++q) {
            if (kb0 + q < g.nkb) {
                uint8_t *d = dst0 + (size_t)(kb0 + q) * g.blk + off;
                convert8(x[q], d, d + kPackPlane, split);
            }
        }
    }
}

// Pack panel p of B^T (columns 128p..128p+127 of B), converter warps 0..7.
// Warp w: 8-wide k chunk w & 1 of every block, columns 32(w >> 1) + lane; the
// eight k rows of a chunk are eight coalesced 128-byte row reads per warp.
__device__ __forceinline__ void gemm_pack_b(const float *__restrict__ B, const PackGeom &g, uint32_t p,
                                            bool split) {
    const uint32_t w = threadIdx.x >> 5, lane = lane_id();
    const uint32_t c = w & 1u, cl = 32 * (w >> 1) + lane, gc = p * kGemmBN + cl, n = g.n;
    const uint32_t off = sw32_offset(cl, c);
    const float *col = B + min(gc, n - 1);
    uint8_t *dst0 = g.b + (size_t)p * g.nkb * g.blk;
    for (uint32_t kb0 = 0; kb0 < g.nkb; kb0 += 4) {
        float x[4][8];
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
            const uint32_t gk = (kb0 + q) * kGemmKB + 8 * c;
#pragma unroll
            for (uint32_t j = 0; j < 8; ++j)
                x[q][j] = (gc < n && gk + j < n) ? __ldg(col + (size_t)(gk + j) * n) : 0.0f;
        }
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
            if (kb0 + q < g.nkb) {
                uint8_t *d = dst0 + (size_t)(kb0 + q) * g.blk + off;
                convert8(x[q], d, d + kPackPlane, split);
            }
        }
    }
}

// ---- staged packing (16-byte aligned rows) ---------------------------------
// cp.async copies (16 bytes per thread, zero-filled past `valid` bytes) into
// a per-warp ring of kPackStages shared-memory stages, so a warp keeps
// kPackStages - 1 slices of 64 k in flight while it converts one.  Each warp
// loads only what it converts, so a __syncwarp orders the stage's reuse.
constexpr uint32_t kPackStages = 5;
constexpr uint32_t kPackApitch = 68;                 // floats per staged A row (conflict-free reads)
constexpr uint32_t kPackWarpStage = 16 * kPackApitch * 4;   // >= 8 k rows x 128 floats of B
static_assert(8 * 128 * 4 <= kPackWarpStage, "a B stage fits a warp's stage");
static_assert(kGemmConvWarps * kPackStages * kPackWarpStage <= kGemmOpsBytes, "pack stages fit the GEMM area");

__device__ __forceinline__ void cp_async16(void *smem, const void *gsrc, uint32_t valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gsrc), "r"(valid)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_stages() {
    asm volatile("cp.async.wait_group %0;" ::"n"(kPackStages - 1) : "memory");
}

// A panel p, 16-byte aligned rows: warp w stages its rows 16w..16w+15 in
// slices of 64 k (lane: row 2q + (lane >> 4), 16-byte chunk lane & 15).
__device__ __forceinline__ void gemm_pack_a_staged(const float *__restrict__ A, const PackGeom &g, uint32_t p,
                                                   bool split, uint8_t *stage_area) {
    const uint32_t w = threadIdx.x >> 5, lane = lane_id(), n = g.n;
    float *st = reinterpret_cast<float *>(stage_area + (size_t)w * kPackStages * kPackWarpStage);
    const uint32_t nsl = (n + 63) / 64;
    auto issue = [&](uint32_t sl) {
        if (sl < nsl) {
            float *buf = st + (sl % kPackStages) * (kPackWarpStage / 4);
#pragma unroll
            for (uint32_t q = 0; q < 8; ++q) {
                const uint32_t rr = 2 * q + (lane >> 4), ch = lane & 15u;
                const uint32_t gr = p * kGemmBM + 16 * w + rr, gk = sl * 64 + 4 * ch;
                const uint32_t valid = (gr < n && gk < n) ? min(16u, (n - gk) * 4) : 0u;
                const float *src = valid ? A + (size_t)gr * n + gk : A;
                cp_async16(buf + rr * kPackApitch + 4 * ch, src, valid);
            }
        }
        cp_async_commit();
    };
    for (uint32_t sl = 0; sl + 1 < kPackStages; ++sl) issue(sl);
    const uint32_t r = 16 * w + (lane & 15u), c = lane >> 4, rl = lane & 15u;
    const uint32_t off = sw32_offset(r, c);
    uint8_t *dst0 = g.a + (size_t)p * g.nkb * g.blk;
    for (uint32_t sl = 0; sl < nsl; ++sl) {
        issue(sl + kPackStages - 1);
        cp_async_wait_stages();
        __syncwarp();
        const float *buf = st + (sl % kPackStages) * (kPackWarpStage / 4) + rl * kPackApitch;
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t kb = 4 * sl + j;
            if (kb < g.nkb) {
                const float4 lo = *reinterpret_cast<const float4 *>(buf + 16 * j + 8 * c);
                const float4 hi = *reinterpret_cast<const float4 *>(buf + 16 * j + 8 * c + 4);
                const float x[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                uint8_t *d = dst0 + (size_t)kb * g.blk + off;
                convert8(x, d, d + kPackPlane, split);
            }
        }
        __syncwarp();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// B^T panel p, 16-byte aligned rows: warp w stages k rows 8w..8w+7 of each
// 64-k slice (128 columns, lane: row q, 16-byte chunk lane) and converts them
// as chunk w & 1 of block w >> 1 of the slice for columns lane + 32i.
__device__ __forceinline__ void gemm_pack_b_staged(const float *__restrict__ B, const PackGeom &g, uint32_t p,
                                                   bool split, uint8_t *stage_area) {
    const uint32_t w = threadIdx.x >> 5, lane = lane_id(), n = g.n;
    float *st = reinterpret_cast<float *>(stage_area + (size_t)w * kPackStages * kPackWarpStage);
    const uint32_t nsl = (n + 63) / 64;
    auto issue = [&](uint32_t sl) {
        if (sl < nsl) {
            float *buf = st + (sl % kPackStages) * (kPackWarpStage / 4);
#pragma unroll
            for (uint32_t q = 0; q < 8; ++q) {
                const uint32_t gk = sl * 64 + 8 * w + q, gc = p * kGemmBN + 4 * lane;
                const uint32_t valid = (gk < n && gc < n) ? min(16u, (n - gc) * 4) : 0u;
                const float *src = valid ? B + (size_t)gk * n + gc : B;
                cp_async16(buf + q * 128 + 4 * lane, src, valid);
            }
        }
        cp_async_commit();
    };
    for (uint32_t sl = 0; sl + 1 < kPackStages; ++sl) issue(sl);
    const uint32_t c = w & 1u, jb = w >> 1;
    uint8_t *dst0 = g.b + (size_t)p * g.nkb * g.blk;
    for (uint32_t sl = 0; sl < nsl; ++sl) {
        issue(sl + kPackStages - 1);
        cp_async_wait_stages();
        __syncwarp();
        const float *buf = st + (sl % kPackStages) * (kPackWarpStage / 4);
        const uint32_t kb = 4 * sl + jb;
        if (kb < g.nkb) {
#pragma unroll
            for (uint32_t i = 0; i < 4; ++i) {
                const uint32_t col = lane + 32 * i;
                float x[8];
#pragma unroll
                for (uint32_t q = 0; q < 8; ++q) x[q] = buf[q * 128 + col];
                uint8_t *d = dst0 + (size_t)kb * g.blk + sw32_offset(col, c);
                convert8(x, d, d + kPackPlane, split);
            }
        }
        __syncwarp();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---- tile sequences ---------------------------------------------------------
constexpr uint32_t kPackTmemCols = 512;   // two accumulator buffers of 256 columns

// One output tile of a packed message.
// A wide tile (BF16 only) covers columns 128 tn .. 128 tn + 255: B panels tn
// and tn + 1, whose k-block planes sit side by side in the slot so that one
// N = 256 MMA reads both.
struct TileRef {
    PackGeom g;
    float *C;
    uint32_t tm, tn;
    bool split;
    bool wide;
};

// Epilogue of a tile from the accumulator buffer at TMEM column `acc`, one
// of warps 4..7: TMEM lanes 32 (w % 4).. (rows), all 128 columns (256 for a
// wide tile); the split form adds columns acc + 128.. to them.  Stores are
// masked at the edge.
__device__ __forceinline__ void packed_epilogue(const TileRef &t, uint32_t tmem, uint32_t acc) {
    const uint32_t lane = lane_id(), q = (threadIdx.x >> 5) & 3u, n = t.g.n;
    const uint32_t gr = t.tm * kGemmBM + 32 * q + lane;
    float *crow = t.C + (size_t)min(gr, n - 1) * n;
    const uint32_t cols = t.wide ? 2 * kGemmBN : kGemmBN;
#pragma unroll 1
    for (uint32_t cc = 0; cc < cols; cc += 32) {
        uint32_t r[32];
        tmem_ld_32x32(tmem + ((32 * q) << 16) + acc + cc, r);
        if (t.split) {
            uint32_t r2[32];
            tmem_ld_32x32(tmem + ((32 * q) << 16) + acc + kGemmBN + cc, r2);
#pragma unroll
            for (uint32_t j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(r2[j]));
        }
        if (gr < n) {
            const uint32_t gc0 = t.tn * kGemmBN + cc;
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
}

// k blocks per slot for tile `r`, and the slots it streams.
__device__ __forceinline__ uint32_t slot_blocks(const TileRef &r) {
    return r.split ? kSlotBlocksSplit : (r.wide ? kSlotBlocksWide : kSlotBlocksNarrow);
}
__device__ __forceinline__ uint32_t packed_slots_of(const TileRef &r) {
    const uint32_t bps = slot_blocks(r);
    return (r.g.nkb + bps - 1) / bps;
}

// Compute `count` output tiles (tile(i): TileRef of the i-th) as one
// pipeline over the whole CTA:
//   * warp 0's lane 0 streams every tile's k blocks into the slot ring (per
//     slot of slot_blocks(r) blocks: one bulk copy of A's blocks, and one of
//     B's, or two per block for a wide tile), running ahead into the
//     next tile while the current one is multiplied;
//   * warp kGemmConvWarps's lane 0 issues the MMAs, alternating between two
//     accumulator buffers (TMEM columns 0.. and 256..) so a tile's MMAs can
//     start while the previous tile's epilogue still reads its buffer;
//   * warps 4..7 run the epilogues, then free the buffer.
// `K` carries the slot and buffer phases across calls (K.pk_uses, K.tiles).
// Waits and commits are per slot: an mbarrier wait costs hundreds of cycles
// even when the phase has completed, more than the MMAs of one k block.
// Returns false if a bounded wait expired.
template <class TileAt, class CtaSync>
__device__ bool gemm_tiles_packed(TileAt tile, uint32_t count, PackedSlots &S, GemmBars &Bb, GemmCounters &K,
                                  uint64_t limit_ns, CtaSync cta_sync) {
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    bool ok = true;
    if (warp == 0 && lane == 0) {
        // the images were written with ordinary stores by the CTAs that ran
        // the pack items (ordered before these tiles by the work queue), and
        // a pack item may have used the slot area through ordinary accesses
        // (ordered by the CTA barrier between items): make both visible to
        // the bulk copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        fence_proxy_async_smem();
        uint32_t u = K.pk_uses;
        for (uint32_t t = 0; t < count && ok; ++t) {
            const TileRef r = tile(t);
            const uint32_t nb = r.g.nkb, bps = slot_blocks(r), ns = packed_slots_of(r);
            const uint8_t *ab = r.g.a + (size_t)r.tm * nb * r.g.blk, *bb = r.g.b + (size_t)r.tn * nb * r.g.blk;
            for (uint32_t i = 0; i < ns; ++i, ++u) {
                const uint32_t s = u % kPackSlots;
                if (u >= kPackSlots) {
                    ok = gemm_wait(&Bb.pk_empty[s], (u / kPackSlots - 1u) & 1u, limit_ns);
                    if (!ok) break;
                }
                const uint32_t k0 = i * bps, kn = min(bps, nb - k0);
                mbar_arrive_expect_tx(&Bb.pk_full[s], (r.wide ? 3 : 2) * kn * r.g.blk);
                bulk_g2s(S.s[s], ab + (size_t)k0 * r.g.blk, kn * r.g.blk, &Bb.pk_full[s]);
                uint8_t *sb = S.s[s] + bps * r.g.blk;
                if (r.wide) {
                    // block b of panels tn and tn + 1, side by side
                    const uint8_t *bb2 = bb + (size_t)nb * r.g.blk;
                    for (uint32_t b = 0; b < kn; ++b) {
                        bulk_g2s(sb + 2 * b * r.g.blk, bb + (size_t)(k0 + b) * r.g.blk, r.g.blk, &Bb.pk_full[s]);
                        bulk_g2s(sb + (2 * b + 1) * r.g.blk, bb2 + (size_t)(k0 + b) * r.g.blk, r.g.blk,
                                 &Bb.pk_full[s]);
                    }
                } else {
                    bulk_g2s(sb, bb + (size_t)k0 * r.g.blk, kn * r.g.blk, &Bb.pk_full[s]);
                }
            }
        }
        // after an expired wait, let the copies in flight land (bounded)
        for (uint32_t q = (u - K.pk_uses > kPackSlots ? u - kPackSlots : K.pk_uses); !ok && q < u; ++q)
            gemm_wait(&Bb.pk_full[q % kPackSlots], (q / kPackSlots) & 1u, limit_ns);
    } else if (warp == kGemmConvWarps && lane == 0) {
        uint32_t u = K.pk_uses, tt = K.tiles;
        for (uint32_t t = 0; t < count && ok; ++t, ++tt) {
            const TileRef r = tile(t);
            const uint32_t nb = r.g.nkb, bps = slot_blocks(r), ns = packed_slots_of(r), bsel = tt & 1u,
                           acc = Bb.tmem + bsel * 256u;
            if (tt >= 2) {
                ok = gemm_wait(&Bb.acc_empty[bsel], ((tt >> 1) - 1u) & 1u, limit_ns);
                if (!ok) break;
            }
            tc_fence_after();
            for (uint32_t i = 0; i < ns; ++i, ++u) {
                const uint32_t s = u % kPackSlots;
                ok = gemm_wait(&Bb.pk_full[s], (u / kPackSlots) & 1u, limit_ns);
                if (!ok) break;
                tc_fence_after();
                const uint32_t kn = min(bps, nb - i * bps);
                const uint8_t *sa = S.s[s], *sb = S.s[s] + bps * r.g.blk;
                if (r.wide) {
                    const uint32_t id256 = gemm_idesc(kGemmBM, 2 * kGemmBN);
                    for (uint32_t b = 0; b < kn; ++b)
                        tc_mma_f16(acc, smem_desc_sw32(sa + b * r.g.blk), smem_desc_sw32(sb + 2 * b * r.g.blk), id256,
                                   (i == 0 && b == 0) ? 0u : 1u);
                } else {
                    for (uint32_t b = 0; b < kn; ++b)
                        gemm_mma_planes(sa + b * r.g.blk, sa + b * r.g.blk + kPackPlane, sb + b * r.g.blk, acc,
                                        r.split, i == 0 && b == 0);
                }
                tc_commit(&Bb.pk_empty[s]);
            }
            tc_commit(&Bb.acc_full[bsel]);
        }
    } else if (warp >= 4 && warp < kGemmConvWarps) {
        uint32_t tt = K.tiles;
        for (uint32_t t = 0; t < count && ok; ++t, ++tt) {
            const TileRef r = tile(t);
            const uint32_t bsel = tt & 1u;
            ok = gemm_wait(&Bb.acc_full[bsel], (tt >> 1) & 1u, limit_ns);
            if (!__all_sync(0xFFFFFFFFu, ok)) {
                ok = false;
                break;
            }
            tc_fence_after();
            packed_epilogue(r, Bb.tmem, bsel * 256u);
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&Bb.acc_empty[bsel]))
                             : "memory");
        }
    }
    if (warp == 0 || warp == kGemmConvWarps) __syncwarp();
    // every thread advances the phase counters the same way
    uint32_t slots = 0;
    for (uint32_t t = 0; t < count; ++t) slots += packed_slots_of(tile(t));
    K.pk_uses += slots;
    K.tiles += count;
    // the next sequence's MMAs overwrite the buffers, and a pack item may
    // reuse the slot area: every epilogue read and MMA must be complete
    tc_fence_before();
    cta_sync();
    tc_fence_after();
    return ok;
}

}  // namespace cafgpu

namespace cafgpu {
static_assert(pack_bytes(kPackSmallMaxN, true) == kPackSmallBytes, "small scratch class holds n <= kPackSmallMaxN");
static_assert(pack_bytes(kMaxDrainGemmN, true) == kPackLargeBytes, "large scratch class holds n <= kMaxDrainGemmN");
}  // namespace cafgpu
