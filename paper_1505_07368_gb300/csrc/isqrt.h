// floor(sqrt(n)) for any 64-bit n, exact, in integer arithmetic only.
//
// The binary digit-by-digit method (Warren, "Hacker's Delight", 2nd ed.,
// Sec. 11-1): the root is built one bit per step from the most significant
// bit down; at each step the candidate bit is kept when the remainder still
// covers it.  At most 32 steps of shifts, adds and compares -- once per
// factorization message, so the device path needs no floating point.
// Compiled for both host and device, so the host's prime-table limit and the
// device's per-message bounds are the same function.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define CAFGPU_HD __host__ __device__ __forceinline__
#else
#define CAFGPU_HD inline
#endif

namespace cafgpu {

CAFGPU_HD uint64_t isqrt_u64(uint64_t n) {
    uint64_t rem = n, root = 0;
    uint64_t bit = 1ull << 62;            // the largest power of four in 64 bits
    while (bit > rem) bit >>= 2;
    while (bit != 0) {
        if (rem >= root + bit) {          // root < 2^32 and bit <= 2^62: no overflow
            rem -= root + bit;
            root = (root >> 1) + bit;
        } else {
            root >>= 1;
        }
        bit >>= 2;
    }
    return root;
}

}  // namespace cafgpu
