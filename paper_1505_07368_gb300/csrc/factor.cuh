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
#include "isqrt.h"

namespace cafgpu {

__device__ __forceinline__ bool mont_divides(uint64_t n, uint32_t nlneg, uint32_t p,
                                             uint32_t pinv, uint32_t plim) {
    uint32_t m0 = nlneg * pinv;
    uint64_t t = (uint64_t)m0 * p + n;
    uint32_t m1 = (uint32_t)(t >> 32) * pinv;
    return m1 <= plim;
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
//
// Per message the warp keeps nl = -n mod 2^32 and ch = floor(n / 2^32) +
// [n mod 2^32 != 0].  Since n + m0*p == 0 (mod 2^32), the high word of the
// 64-bit sum is umulhi(m0, p) + ch exactly, so the test needs only 32-bit
// multiplies: m0 = nl*pinv, n1 = umulhi(m0, p) + ch, m1 = n1*pinv, m1 <= plim.
// ---------------------------------------------------------------------------
struct SweepRegs {
    uint32_t nl[kFactorKMax];
    uint32_t ch[kFactorKMax];
    uint64_t ids;               // 4 bits per slot: message index in the batch
    int k;
};

// Slots at index >= k hold n = 1, which no prime divides, so the test can
// run over whole blocks of slots without checking k per slot.
constexpr uint32_t kDummyNl = 0xFFFFFFFFu;   // -1 mod 2^32
constexpr uint32_t kDummyCh = 1u;            // 0 + [1 != 0]

__device__ __forceinline__ void sweep_init(SweepRegs &s) {
    s.k = 0;
    s.ids = 0;
#pragma unroll
    for (int j = 0; j < (int)kFactorKMax; ++j) {
        s.nl[j] = kDummyNl;
        s.ch[j] = kDummyCh;
    }
}

__device__ __forceinline__ uint32_t slot_id(const SweepRegs &s, int j) {
    return (uint32_t)(s.ids >> (4 * j)) & 15u;
}

__device__ __forceinline__ void sweep_set(SweepRegs &s, int i, uint64_t n) {
    const uint32_t lo = (uint32_t)n;
    s.nl[i] = 0u - lo;
    s.ch[i] = (uint32_t)(n >> 32) + (lo != 0u ? 1u : 0u);
}

// Remove slot p (0 <= p < k) keeping the others in order; the last slot
// becomes a dummy.
__device__ __forceinline__ void sweep_remove(SweepRegs &s, int p) {
#pragma unroll
    for (int i = 0; i < (int)kFactorKMax - 1; ++i) {
        if (i >= p) {
            s.nl[i] = s.nl[i + 1];
            s.ch[i] = s.ch[i + 1];
        }
    }
    s.nl[kFactorKMax - 1] = kDummyNl;
    s.ch[kFactorKMax - 1] = kDummyCh;
    const uint64_t low = (p == 0) ? 0ull : (s.ids & ((1ull << (4 * p)) - 1ull));
    const uint64_t high = (p >= 15) ? 0ull : ((s.ids >> (4 * (p + 1))) << (4 * p));
    s.ids = low | high;
    --s.k;
}

__device__ __forceinline__ bool sweep_test(const SweepRegs &s, int j, uint32_t p, uint32_t pinv, uint32_t plim) {
    const uint32_t m0 = s.nl[j] * pinv;
    const uint32_t n1 = __umulhi(m0, p) + s.ch[j];
    return n1 * pinv <= plim;
}

// Slots B, B+1 against NP primes per lane (one per chunk): 2 NP independent
// multiply chains; a hit is the smaller m1 at or below the limit.
template <int B, int NP>
__device__ __forceinline__ bool sweep_block(const SweepRegs &s, const uint32_t (&p)[NP], const uint32_t (&pi)[NP],
                                            const uint32_t (&pl)[NP]) {
    uint32_t a[NP][2];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
        for (int i = 0; i < 2; ++i) a[q][i] = s.nl[B + i] * pi[q];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
        for (int i = 0; i < 2; ++i) a[q][i] = __umulhi(a[q][i], p[q]) + s.ch[B + i];
    bool hit = false;
#pragma unroll
    for (int q = 0; q < NP; ++q) hit |= min(a[q][0] * pi[q], a[q][1] * pi[q]) <= pl[q];
    return hit;
}

static_assert(kFactorKMax == 16, "sweep_chunks unrolls 16 slots in blocks of two");

// True if any held message is divisible by any of this lane's NP primes.
// Slots at index >= k hold n = 1, so only whole blocks of two are tested.
template <int NP>
__device__ __forceinline__ bool sweep_chunks(const SweepRegs &s, const uint32_t (&p)[NP], const uint32_t (&pi)[NP],
                                             const uint32_t (&pl)[NP]) {
    bool hit = false;
    switch ((s.k + 1) >> 1) {
        case 8: hit |= sweep_block<14, NP>(s, p, pi, pl); [[fallthrough]];
        case 7: hit |= sweep_block<12, NP>(s, p, pi, pl); [[fallthrough]];
        case 6: hit |= sweep_block<10, NP>(s, p, pi, pl); [[fallthrough]];
        case 5: hit |= sweep_block<8, NP>(s, p, pi, pl); [[fallthrough]];
        case 4: hit |= sweep_block<6, NP>(s, p, pi, pl); [[fallthrough]];
        case 3: hit |= sweep_block<4, NP>(s, p, pi, pl); [[fallthrough]];
        case 2: hit |= sweep_block<2, NP>(s, p, pi, pl); [[fallthrough]];
        case 1: hit |= sweep_block<0, NP>(s, p, pi, pl); break;
        default: break;
    }
    return hit;
}

// Bit j set if this lane's prime divides the message in slot j (slow path,
// run only for chunks where some lane hit).
__device__ __forceinline__ uint32_t sweep_which(const SweepRegs &s, uint32_t p, uint32_t pinv, uint32_t plim) {
    uint32_t hits = 0;
#pragma unroll
    for (int j = 0; j < (int)kFactorKMax; ++j)
        if (j < s.k && sweep_test(s, j, p, pinv, plim)) hits |= 1u << j;
    return hits;
}

}  // namespace cafgpu
