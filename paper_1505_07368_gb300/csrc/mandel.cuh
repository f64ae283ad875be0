// Mandelbrot escape counts: the payload of the paper's OpenCL actor
// experiment (Sec. 5, "Integrating OpenCL Actors": a 1920 x 1080 image of a
// cut of the complex plane with 120 or 1200 maximum iterations).
//
// The count of c is the number of updates z <- z^2 + c, from z = 0, made
// before |z|^2 > 4 is first seen, at most max_iter.  Every step is one float32
// operation rounded to nearest, written with the _rn intrinsics so that no
// multiply and add are fused:
//
//   x2 = zr*zr; y2 = zi*zi; stop if x2 + y2 > 4;
//   xy = zr*zi; zi = (xy + xy) + cy; zr = (x2 - y2) + cx.
//
// That makes the count a pure function of (cx, cy, max_iter), equal bit for
// bit on any IEEE float32 machine that follows the same order.
//
// The loop runs blocks of kU updates with no branch between them, folding
// the escape tests into one predicate (kU = 16 for max_iter >= 512, else 12:
// a longer block amortises the loop, a shorter one wastes fewer updates after
// an escape and leaves a shorter one-at-a-time tail; both are exact).  A block in which some test
// fired is repeated from its saved start one update at a time, so the count
// is the same as with a test before every update.  After an escape the block
// may overflow to inf or NaN; the predicate already holds then (a NaN test is
// false but cannot clear it), and the repeat starts from the saved, finite z.
#pragma once

#include <cuda_runtime.h>

#include "layout.h"

namespace cafgpu {

// One update of z with its escape test folded into `esc` (no branch).
__device__ __forceinline__ void mandel_step(float &zr, float &zi, float cx, float cy, bool &esc) {
    const float x2 = __fmul_rn(zr, zr);
    const float y2 = __fmul_rn(zi, zi);
    esc |= __fadd_rn(x2, y2) > 4.0f;
    const float xy = __fmul_rn(zr, zi);
    zi = __fadd_rn(__fadd_rn(xy, xy), cy);
    zr = __fadd_rn(__fsub_rn(x2, y2), cx);
}

// The count of c from state z after k updates, testing before each update:
// used on the block that escaped, and on the last max_iter % unroll updates.
__device__ __forceinline__ uint32_t mandel_single(float zr, float zi, float cx, float cy, uint32_t k,
                                                  uint32_t max_iter) {
    while (k < max_iter) {
        const float x2 = __fmul_rn(zr, zr);
        const float y2 = __fmul_rn(zi, zi);
        if (__fadd_rn(x2, y2) > 4.0f) break;
        const float xy = __fmul_rn(zr, zi);
        zi = __fadd_rn(__fadd_rn(xy, xy), cy);
        zr = __fadd_rn(__fsub_rn(x2, y2), cx);
        ++k;
    }
    return k;
}

template <uint32_t kU>
__device__ __forceinline__ uint32_t mandel_count_blocks(float cx, float cy, uint32_t max_iter) {
    float zr = 0.0f, zi = 0.0f;
    uint32_t k = 0;
    while (k + kU <= max_iter) {
        const float sr = zr, si = zi;
        bool esc = false;
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) mandel_step(zr, zi, cx, cy, esc);
        if (esc) {
            zr = sr;
            zi = si;
            break;
        }
        k += kU;
    }
    return mandel_single(zr, zi, cx, cy, k, max_iter);
}

// max_iter is the same for every pixel of a job, so the choice does not diverge.
__device__ __forceinline__ uint32_t mandel_count(float cx, float cy, uint32_t max_iter) {
    return max_iter >= 512 ? mandel_count_blocks<16>(cx, cy, max_iter) : mandel_count_blocks<12>(cx, cy, max_iter);
}

// c of pixel p of a job (row-major over its rows): one rounded product and
// one rounded sum per coordinate.  width and row0 + rows are below 2^24, so
// the integer coordinates convert to float32 exactly.
__device__ __forceinline__ void mandel_c(const MandelDesc &d, uint32_t p, float &cx, float &cy) {
    const uint32_t r = p / d.width;
    const uint32_t i = p - r * d.width;
    cx = __fadd_rn(d.x0, __fmul_rn(__uint2float_rn(i), d.dx));
    cy = __fadd_rn(d.y0, __fmul_rn(__uint2float_rn(d.row0 + r), d.dy));
}

// A descriptor the library accepts (checked on the host for host messages and
// on the device for device batches).
__host__ __device__ __forceinline__ bool mandel_desc_ok(const MandelDesc &d) {
    const uint64_t pixels = (uint64_t)d.width * d.rows;
    return d.out != 0 && (d.out & 3u) == 0 && d.width > 0 && d.rows > 0 && pixels <= kMandelMaxPixels &&
           d.width <= kMandelMaxCoord && (uint64_t)d.row0 + d.rows <= kMandelMaxCoord && d.max_iter <= kMandelMaxIter;
}

}  // namespace cafgpu
