// Factorization payload: exact trial division of a 64-bit n by the odd primes
// p with p*p <= n, in increasing order, the first hit giving (p, n/p).  This
// is the numeric side load of the paper's mixed benchmark (Sec. 5, "Mixed
// Operations Under Work Load"); the smallest divisor >= 2 of n is always
// prime, so dividing by primes only returns the same pair as dividing by
// every integer.
//
// Divisibility test (Montgomery, "Modular multiplication without trial
// division", Math. Comp. 44, 1985, REDC applied twice with 32-bit limbs; the
// final test is the exact-division check of Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994):
//
//   p odd, p < 2^31, n < 2^62, pinv = p^-1 mod 2^32, plim = floor((2^32-1)/p)
//   m0 = (-n mod 2^32) * pinv  mod 2^32   ->  n + m0*p == 0 (mod 2^32)
//   t  = n + m0*p                          (< 2^62 + 2^63, no overflow)
//   n1 = t / 2^32                          (exact, < 2^32; p | n  <=>  p | n1)
//   m1 = n1 * pinv mod 2^32                ->  p | n1  <=>  m1 <= plim
//
// Three 32-bit integer multiplies and one compare per (n, p) pair; the
// per-prime constants pinv and plim come from the prime table.
#pragma once

#include "common.cuh"

namespace cafgpu {

__device__ __forceinline__ bool mont_divides(uint64_t n, uint32_t nlneg, uint32_t p,
                                             uint32_t pinv, uint32_t plim) {
    uint32_t m0 = nlneg * pinv;
    uint64_t t = (uint64_t)m0 * p + n;
    uint32_t m1 = (uint32_t)(t >> 32) * pinv;
    return m1 <= plim;
}

// floor(sqrt(n)) for n < 2^62, exact.
__device__ __forceinline__ uint64_t isqrt_u64(uint64_t n) {
    uint64_t s = (uint64_t)sqrt((double)n);
    while (s * s > n) --s;
    while ((s + 1) * (s + 1) <= n) ++s;
    return s;
}

// Number of table primes <= x (table sorted increasingly, odd primes).
__device__ __forceinline__ uint32_t primes_le(const uint32_t *primes, uint32_t nprimes, uint64_t x) {
    uint32_t lo = 0, hi = nprimes;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(primes + mid) <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Bound for message n: odd primes p with p*p <= n (0 if trivial: n < 9).
__device__ __forceinline__ uint32_t factor_bound(const uint32_t *primes, uint32_t nprimes, uint64_t n) {
    if (n < 9) return 0;
    return primes_le(primes, nprimes, isqrt_u64(n));
}

// Reply for one message once the sweep is over.  found = index of the first
// dividing odd prime (kNoFactor if none), bound = factor_bound(n).
__device__ __forceinline__ void factor_result(uint64_t n, bool even, uint32_t found, uint32_t bound,
                                              const uint32_t *primes, int32_t *status,
                                              uint64_t *r0, uint64_t *r1) {
    if (even && n >= 4) {
        *status = 0;
        *r0 = 2;
        *r1 = n >> 1;
    } else if (found < bound) {
        uint64_t p = __ldg(primes + found);
        *status = 0;
        *r0 = p;
        *r1 = n / p;
    } else {
        *status = 1;
        *r0 = 1;
        *r1 = n;
    }
}

__device__ __forceinline__ void write_reply(uint64_t addr, int32_t status, uint64_t r0, uint64_t r1,
                                            uint64_t /*tag*/, uint32_t token) {
    if (!addr) return;
    Reply *r = reinterpret_cast<Reply *>(addr);
    r->status = status;
    r->r0 = r0;
    r->r1 = r1;
    r->t_done = globaltimer();
    st_release_sys(&r->done, token);
}

// ---------------------------------------------------------------------------
// Batched sweep.  A warp holds the still-undecided messages of a batch in
// registers, compacted to slots 0..k-1; each lane takes one prime of a chunk
// of 32 consecutive table primes and tests it against every held message.
// A message leaves the warp when a lane finds a divisor (the smallest index
// among the lanes of that chunk is the first divisor, because the chunks run
// in increasing order), when its bound is passed, or when another warp has
// recorded a divisor below the current position.
// ---------------------------------------------------------------------------
struct SweepRegs {
    uint64_t n[kFactorKMax];
    uint32_t nl[kFactorKMax];   // -n mod 2^32
    uint64_t ids;               // 4 bits per slot: message index in the batch
    int k;
};

__device__ __forceinline__ uint32_t slot_id(const SweepRegs &s, int j) {
    return (uint32_t)(s.ids >> (4 * j)) & 15u;
}

// Remove slot p (0 <= p < k) keeping the others in order.
__device__ __forceinline__ void sweep_remove(SweepRegs &s, int p) {
#pragma unroll
    for (int i = 0; i < (int)kFactorKMax - 1; ++i) {
        if (i >= p) {
            s.n[i] = s.n[i + 1];
            s.nl[i] = s.nl[i + 1];
        }
    }
    const uint64_t low = (p == 0) ? 0ull : (s.ids & ((1ull << (4 * p)) - 1ull));
    const uint64_t high = (p >= 15) ? 0ull : ((s.ids >> (4 * (p + 1))) << (4 * p));
    s.ids = low | high;
    --s.k;
}

#define CAFGPU_TEST_SLOT(J)                                                  \
    case (J) + 1: {                                                          \
        uint32_t m0 = s.nl[J] * pinv;                                        \
        uint64_t t = (uint64_t)m0 * p + s.n[J];                              \
        uint32_t m1 = (uint32_t)(t >> 32) * pinv;                            \
        hits |= (m1 <= plim) ? (1u << (J)) : 0u;                             \
    }

// Test the 32 primes at [c, c+32) (one per lane) against slots 0..k-1.
__device__ __forceinline__ uint32_t sweep_chunk(const SweepRegs &s, uint32_t p, uint32_t pinv,
                                                uint32_t plim) {
    uint32_t hits = 0;
    switch (s.k) {
        CAFGPU_TEST_SLOT(15)
        CAFGPU_TEST_SLOT(14)
        CAFGPU_TEST_SLOT(13)
        CAFGPU_TEST_SLOT(12)
        CAFGPU_TEST_SLOT(11)
        CAFGPU_TEST_SLOT(10)
        CAFGPU_TEST_SLOT(9)
        CAFGPU_TEST_SLOT(8)
        CAFGPU_TEST_SLOT(7)
        CAFGPU_TEST_SLOT(6)
        CAFGPU_TEST_SLOT(5)
        CAFGPU_TEST_SLOT(4)
        CAFGPU_TEST_SLOT(3)
        CAFGPU_TEST_SLOT(2)
        CAFGPU_TEST_SLOT(1)
        CAFGPU_TEST_SLOT(0)
        default:
            break;
    }
    return hits;
}
#undef CAFGPU_TEST_SLOT
static_assert(kFactorKMax == 16, "sweep_chunk unrolls 16 slots");

}  // namespace cafgpu
