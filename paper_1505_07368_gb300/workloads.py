"""Seeded synthetic inputs for the GPU compute-actor workloads.

This module only draws inputs: random numbers, random primes, message
lists and arrival times.  It holds none of the computation the actors
perform (no trial division, no matrix product), so both the CUDA path and
the CPU oracle can take their inputs from it without sharing any of the
method's arithmetic.

Randomness is the counter-based SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
output i of a stream is the SplitMix64 finaliser applied to
``key + (i + 1) * 0x9E3779B97F4A7C15``.  Everything is plain numpy uint64
arithmetic, so the same seed gives the same integers on x86-64 and on
AArch64.  Floating-point draws (normals, log-uniform sizes) go through
numpy's float64 ``log``/``exp``/``cos``; those can differ in the last ulp
between platforms, which moves a value by at most one ulp.

The five workloads follow the evaluation setups of the paper (Sec. 5,
"Mixed Operations Under Work Load" and "Integrating OpenCL Actors") as
restated for a single GPU:

* ``config1``: one actor, 256 semiprimes with prime factors uniform in
  [2^16, 2^20);
* ``config2``: 1024 actors, geometric mailbox lengths (mean 64),
  semiprimes with factors in [2^24, 2^28);
* ``config3``: 256 actors, 4096 square FP32 GEMM messages,
  n uniform in {64, 128, ..., 1024}, N(0,1) entries;
* ``config4``: 64 token rings of 128 actors plus one factorization
  worker per ring, semiprimes with factors in [2^30, 2^31);
* ``config5``: open-loop Poisson arrivals, 70 % factorization
  (log-uniform factors in [2^16, 2^31)) and 30 % split-BF16x3 GEMM
  (n log-uniform in [32, 2048]);
* ``mandel_image`` / ``mandel_slices``: the geometry of the OpenCL actor
  experiment's Mandelbrot image (1920 x 1080 pixels over the cut
  [-0.5 - 0.7375i, 0.1 - 0.1375i]) and its split into row slices.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 150507368

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# message kinds (mirror the C header's CAF_GPU_KIND_* values)
KIND_FACTOR = 1
KIND_GEMM_BF16 = 2
KIND_GEMM_SPLIT = 3
KIND_TOKEN = 4


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of an independent sub-stream ``stream`` of ``seed``."""
    with np.errstate(over="ignore"):
        a = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        b = np.array([(stream * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        return _mix(_mix(a) ^ b)[0]


def u64(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the stream with ``key``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(key) + idx * _GOLDEN)


def uniform01(key, start, count) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(key, start, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def uniform_open(key, start, count) -> np.ndarray:
    """Doubles in (0, 1]."""
    return ((u64(key, start, count) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def normal_f32(key, start, count) -> np.ndarray:
    """N(0,1) float32 by the Box-Muller transform (pairs of draws)."""
    half = (count + 1) // 2
    u1 = uniform_open(key, 2 * start, half)
    u2 = uniform01(key, 2 * start + half, half)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    out = np.empty(2 * half, dtype=np.float64)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count].astype(np.float32)


def bounded(key, start, count, lo: int, hi: int) -> np.ndarray:
    """Integers in [lo, hi) by 32x32 multiply-shift of the high word (hi-lo < 2^32)."""
    span = hi - lo
    assert 0 < span <= (1 << 32)
    z = u64(key, start, count) >> np.uint64(32)
    return (np.uint64(lo) + ((z * np.uint64(span)) >> np.uint64(32))).astype(np.uint64)


# --- primality of sampled candidates (input generation only) -------------

def _powmod(a: np.ndarray, e: np.ndarray, n: np.ndarray) -> np.ndarray:
    # valid for n < 2^32: every product stays below 2^64
    result = np.ones_like(n)
    a = a % n
    e = e.copy()
    while np.any(e):
        odd = (e & np.uint64(1)).astype(bool)
        result = np.where(odd, (result * a) % n, result)
        a = (a * a) % n
        e >>= np.uint64(1)
    return result


def is_prime_u32(n: np.ndarray) -> np.ndarray:
    """Deterministic Miller-Rabin for n < 2^32 with bases 2, 3, 5, 7
    (exact below 3,215,031,751; Jaeschke 1993)."""
    n = np.asarray(n, dtype=np.uint64)
    assert n.size == 0 or int(n.max()) < (1 << 32)
    res = n >= 2
    small = np.array([2, 3, 5, 7], dtype=np.uint64)
    for s in small:
        res &= ~((n % s == 0) & (n != s))
    big = n > 7
    d = n - np.uint64(1)
    r = np.zeros_like(n)
    while True:
        ev = big & (d > 0) & ((d & np.uint64(1)) == 0)
        if not np.any(ev):
            break
        d = np.where(ev, d >> np.uint64(1), d)
        r = np.where(ev, r + np.uint64(1), r)
    nn = np.where(big, n, np.uint64(11))
    dd = np.where(big, d, np.uint64(5))
    for a in small:
        x = _powmod(np.full_like(nn, a), dd, nn)
        ok = (x == 1) | (x == nn - np.uint64(1))
        for i in range(1, int(r.max()) if r.size else 0):
            x = (x * x) % nn
            ok |= (x == nn - np.uint64(1)) & (np.uint64(i) < r)
        res &= ok | ~big
    return res


_SIEVE_PRIMES = np.array([2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47,
                          53, 59, 61, 67, 71, 73, 79, 83, 89, 97], dtype=np.uint64)


def _is_prime_fast(c: np.ndarray) -> np.ndarray:
    # cheap pre-filter by small primes, Miller-Rabin on the survivors
    keep = np.ones(c.shape, bool)
    for s in _SIEVE_PRIMES:
        keep &= (c % s != 0) | (c == s)
    res = np.zeros(c.shape, bool)
    idx = np.nonzero(keep)[0]
    res[idx] = is_prime_u32(c[idx])
    return res


def _primes_from(cand_fn, key, count: int) -> np.ndarray:
    out = []
    have = 0
    pos = 0
    block = max(4096, 24 * count)
    while have < count:
        c = cand_fn(key, pos, block)
        pos += block
        p = c[_is_prime_fast(c)]
        out.append(p)
        have += p.size
    return np.concatenate(out)[:count].astype(np.uint64)


def primes_uniform(key, count: int, lo: int, hi: int) -> np.ndarray:
    """The first ``count`` primes among uniform candidates in [lo, hi)
    (rejection sampling: uniform over the primes of the interval)."""
    return _primes_from(lambda k, s, c: bounded(k, s, c, lo, hi), key, count)


def primes_loguniform(key, count: int, lo: int, hi: int) -> np.ndarray:
    """Primes from x = floor(exp(U[ln lo, ln hi))), composites rejected."""
    a, b = math.log(lo), math.log(hi)

    def cand(k, s, c):
        x = np.floor(np.exp(a + uniform01(k, s, c) * (b - a))).astype(np.uint64)
        return np.clip(x, lo, hi - 1).astype(np.uint64)

    return _primes_from(cand, key, count)


def semiprimes(primes: np.ndarray):
    """Pair consecutive primes: n_i = p_{2i} * p_{2i+1}; returns (n, p, q) with p <= q."""
    a = primes[0::2]
    b = primes[1::2]
    m = min(a.size, b.size)
    a, b = a[:m], b[:m]
    p = np.minimum(a, b)
    q = np.maximum(a, b)
    return p * q, p, q


def geometric(key, count: int, mean: float) -> np.ndarray:
    """Geometric on {1, 2, ...} with success probability 1/mean (inversion)."""
    u = uniform_open(key, 0, count)
    return (1 + np.floor(np.log(u) / math.log1p(-1.0 / mean))).astype(np.int64)


# --- message lists ---------------------------------------------------------

@dataclasses.dataclass
class FactorWorkload:
    """Factorization messages: message i goes to ``actor[i]`` carrying ``n[i]``.

    ``sender``/``sender_seq`` label the producer of each message; the list
    order is the send order.  ``p``/``q`` are the generator's own factors
    (p <= q), usable as a certificate at sizes where the oracle's trial
    division is too slow.
    """
    name: str
    n_actors: int
    actor: np.ndarray
    n: np.ndarray
    p: np.ndarray
    q: np.ndarray
    sender: np.ndarray
    sender_seq: np.ndarray

    @property
    def count(self) -> int:
        return int(self.n.size)


def _label_senders(count: int, n_senders: int):
    sender = (np.arange(count) % n_senders).astype(np.uint32)
    sender_seq = (np.arange(count) // n_senders).astype(np.uint32)
    return sender, sender_seq


def config1(seed: int = SEED_BASE + 1) -> FactorWorkload:
    """1 actor, 256 semiprimes, factors uniform primes in [2^16, 2^20)."""
    k = stream_key(seed, 1)
    n, p, q = semiprimes(primes_uniform(k, 512, 1 << 16, 1 << 20))
    sender, seq = _label_senders(n.size, 1)
    return FactorWorkload("config1", 1, np.zeros(n.size, np.uint32), n, p, q, sender, seq)


def config2(seed: int = SEED_BASE + 2, n_actors: int = 1024, mean_len: float = 64.0,
            lo: int = 1 << 24, hi: int = 1 << 28, n_senders: int = 8,
            max_messages: int | None = None) -> FactorWorkload:
    """1024 actors with geometric(mean 64) mailbox lengths; factors in [2^24, 2^28).

    The send order is a seeded shuffle of the per-actor message multiset;
    messages are labelled with ``n_senders`` round-robin sender ids.
    ``max_messages`` truncates the list (smaller parity cases).
    """
    lens = geometric(stream_key(seed, 2), n_actors, mean_len)
    actor = np.repeat(np.arange(n_actors, dtype=np.uint32), lens)
    # Fisher-Yates with the counter stream: deterministic on any platform
    r = u64(stream_key(seed, 3), 0, actor.size)
    for i in range(actor.size - 1, 0, -1):
        j = int(r[i] % np.uint64(i + 1))
        actor[i], actor[j] = actor[j], actor[i]
    if max_messages is not None:
        actor = actor[:max_messages]
    count = actor.size
    n, p, q = semiprimes(primes_uniform(stream_key(seed, 4), 2 * count, lo, hi))
    sender, seq = _label_senders(count, n_senders)
    return FactorWorkload("config2", n_actors, actor, n, p, q, sender, seq)


@dataclasses.dataclass
class GemmWorkload:
    """GEMM messages over a shared pool of N(0,1) floats.

    Message i multiplies the n_i x n_i row-major matrices stored at
    ``pool[a_off[i]:a_off[i]+n_i^2]`` and ``pool[b_off[i]:...]``; offsets are
    multiples of 4 elements (16 bytes).  Every entry of the pool is an
    independent N(0,1) draw, so each view is a matrix of N(0,1) entries.
    """
    name: str
    n_actors: int
    actor: np.ndarray
    size: np.ndarray
    a_off: np.ndarray
    b_off: np.ndarray
    kind: np.ndarray
    pool_elems: int
    pool_seed: int

    @property
    def count(self) -> int:
        return int(self.size.size)

    def pool(self) -> np.ndarray:
        return gemm_pool(self.pool_seed, self.pool_elems)


def gemm_pool(seed: int, elems: int) -> np.ndarray:
    k = stream_key(seed, 7)
    out = np.empty(elems, dtype=np.float32)
    chunk = 1 << 22
    for s in range(0, elems, chunk):
        c = min(chunk, elems - s)
        out[s:s + c] = normal_f32(k, s, c)
    return out


def _offsets(key, sizes: np.ndarray, pool_elems: int) -> np.ndarray:
    need = sizes.astype(np.int64) ** 2
    span = np.maximum(pool_elems - need, 0) // 4 + 1
    r = u64(key, 0, sizes.size)
    return ((r % span.astype(np.uint64)).astype(np.int64) * 4).astype(np.int64)


def config3(seed: int = SEED_BASE + 3, n_messages: int = 4096, n_actors: int = 256,
            sizes=None, pool_elems: int = 1 << 28, split: bool = False) -> GemmWorkload:
    """256 actors, 4096 GEMM messages, n uniform in {64, 128, ..., 1024}."""
    if sizes is None:
        sizes = (64 * (1 + (u64(stream_key(seed, 5), 0, n_messages) % np.uint64(16)))).astype(np.int64)
    else:
        sizes = np.asarray(sizes, dtype=np.int64)
    n_messages = sizes.size
    assert pool_elems >= int(sizes.max()) ** 2
    actor = (u64(stream_key(seed, 6), 0, n_messages) % np.uint64(n_actors)).astype(np.uint32)
    a_off = _offsets(stream_key(seed, 8), sizes, pool_elems)
    b_off = _offsets(stream_key(seed, 9), sizes, pool_elems)
    kind = np.full(n_messages, KIND_GEMM_SPLIT if split else KIND_GEMM_BF16, np.uint32)
    return GemmWorkload("config3", n_actors, actor, sizes, a_off, b_off, kind, pool_elems, seed)


@dataclasses.dataclass
class RingWorkload:
    """Token rings: ``n_rings`` rings of ``ring_len`` actors, one factor worker per ring.

    ``n[r, k]`` is the k-th semiprime the master of ring r sends to its worker.
    """
    name: str
    n_rings: int
    ring_len: int
    token: int
    n: np.ndarray
    p: np.ndarray
    q: np.ndarray


def ring_rounds(ring_len: int, token: int) -> int:
    """Factor messages per ring: one at start plus one per token receipt with v > 0
    at the master (deliveries k = ring_len, 2*ring_len, ... carry token + 1 - k)."""
    return 1 + sum(1 for k in range(ring_len, token + 1, ring_len) if token + 1 - k > 0)


def config4(seed: int = SEED_BASE + 4, n_rings: int = 64, ring_len: int = 128,
            token: int = 1000, lo: int = 1 << 30, hi: int = 1 << 31) -> RingWorkload:
    rounds = ring_rounds(ring_len, token)
    n, p, q = semiprimes(primes_uniform(stream_key(seed, 10), 2 * n_rings * rounds, lo, hi))
    shape = (n_rings, rounds)
    return RingWorkload("config4", n_rings, ring_len, token,
                        n.reshape(shape), p.reshape(shape), q.reshape(shape))


@dataclasses.dataclass
class ServingWorkload:
    """Open-loop arrivals.  Request i arrives at ``t[i]`` seconds; ``kind[i]`` is
    KIND_FACTOR (payload ``n[i]``) or KIND_GEMM_SPLIT (size ``size[i]``,
    operands at ``a_off``/``b_off`` in the pool)."""
    name: str
    t: np.ndarray
    kind: np.ndarray
    actor: np.ndarray
    n: np.ndarray
    p: np.ndarray
    q: np.ndarray
    size: np.ndarray
    a_off: np.ndarray
    b_off: np.ndarray
    pool_elems: int
    pool_seed: int

    @property
    def count(self) -> int:
        return int(self.t.size)


def config5(seed: int = SEED_BASE + 5, n_requests: int = 1_000_000, rate: float = 1e5,
            frac_factor: float = 0.7, n_factor_actors: int = 2048, n_gemm_actors: int = 1024,
            pool_elems: int = 1 << 24, max_gemm: int = 2048, factor_lo: int = 1 << 16,
            factor_hi: int = 1 << 31) -> ServingWorkload:
    """Open-loop serving mix: Poisson arrivals at `rate`/s, `frac_factor` factorization
    requests (log-uniform prime factors in [factor_lo, factor_hi)), the rest split-BF16x3
    GEMMs with n log-uniform in [32, max_gemm].  Smaller ranges give the parity cases."""
    gaps = -np.log(uniform_open(stream_key(seed, 11), 0, n_requests)) / rate
    t = np.cumsum(gaps)
    is_factor = uniform01(stream_key(seed, 12), 0, n_requests) < frac_factor
    nf = int(is_factor.sum())
    ng = n_requests - nf
    nn, pp, qq = semiprimes(primes_loguniform(stream_key(seed, 13), 2 * nf, factor_lo, factor_hi))
    a, b = math.log(32), math.log(max_gemm)
    sizes = np.rint(np.exp(a + uniform01(stream_key(seed, 14), 0, ng) * (b - a))).astype(np.int64)
    sizes = np.clip(sizes, 32, max_gemm)
    pool_elems = max(pool_elems, max_gemm * max_gemm)
    kind = np.where(is_factor, KIND_FACTOR, KIND_GEMM_SPLIT).astype(np.uint32)
    act_f = (u64(stream_key(seed, 15), 0, n_requests) % np.uint64(n_factor_actors)).astype(np.uint32)
    act_g = (n_factor_actors + u64(stream_key(seed, 16), 0, n_requests) % np.uint64(n_gemm_actors)).astype(np.uint32)
    actor = np.where(is_factor, act_f, act_g).astype(np.uint32)
    n = np.zeros(n_requests, np.uint64)
    p = np.zeros(n_requests, np.uint64)
    q = np.zeros(n_requests, np.uint64)
    n[is_factor], p[is_factor], q[is_factor] = nn, pp, qq
    size = np.zeros(n_requests, np.int64)
    size[~is_factor] = sizes
    a_off = np.zeros(n_requests, np.int64)
    b_off = np.zeros(n_requests, np.int64)
    a_off[~is_factor] = _offsets(stream_key(seed, 17), sizes, pool_elems)
    b_off[~is_factor] = _offsets(stream_key(seed, 18), sizes, pool_elems)
    return ServingWorkload("config5", t, kind, actor, n, p, q, size, a_off, b_off,
                           pool_elems, seed)


def integer_matrix(key, n: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """n x n float32 matrix of integers in [lo, hi] (exact in BF16)."""
    v = bounded(key, 0, n * n, 0, hi - lo + 1).astype(np.int64) + lo
    return v.astype(np.float32).reshape(n, n)


# ---- the OpenCL actor experiment (Sec. 5, "Integrating OpenCL Actors") ----
MANDEL_WIDTH, MANDEL_HEIGHT = 1920, 1080
MANDEL_AREA = (-0.5, -0.7375, 0.1, -0.1375)      # (re min, im min, re max, im max)
MANDEL_ITERS = (120, 1200)                       # the small and the large problem


def mandel_image(width: int = MANDEL_WIDTH, height: int = MANDEL_HEIGHT, area=MANDEL_AREA):
    """(x0, y0, dx, dy) as float32 values: pixel (i, j) lies at c = (x0 + i dx) + (y0 + j dy) i,
    so the `width` x `height` pixels tile `area` from its lower-left corner."""
    re0, im0, re1, im1 = area
    f = np.float32
    return f(re0), f(im0), f((re1 - re0) / width), f((im1 - im0) / height)


def mandel_slices(height: int, parts: int):
    """Split rows 0 .. height-1 into `parts` contiguous slices of near-equal size: [(row0, rows)]."""
    edges = [(height * k) // parts for k in range(parts + 1)]
    return [(edges[k], edges[k + 1] - edges[k]) for k in range(parts) if edges[k + 1] > edges[k]]
