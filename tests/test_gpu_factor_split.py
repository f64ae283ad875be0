"""Split factor batches (the factor_split setting): a large batch is cut into
segments of every S-th table tile, swept by idle teams in other CTAs.  Replies
must be identical to the unsplit sweep's: the smallest divisor (bit-exact
against the generator's factors and the oracle), or no divisor for primes."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch, host_requests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt_split():
    # prime table to 2^31: numbers up to 2^62 - 1
    with C.Runtime(max_actors=8, factor_split=32) as rt:
        a = rt.spawn(C.FACTOR_U64)
        yield rt, a


@pytest.mark.parametrize("k", [1, 3, 16])
def test_large_semiprimes_split(rt_split, k):
    """Factors in [2^30, 2^31) (config 4's range): sweeps of ~25,000 tiles."""
    rt, a = rt_split
    n, p, q = W.semiprimes(W.primes_uniform(W.stream_key(4242, k), 2 * k, 1 << 30, 1 << 31))
    rep = host_requests(rt, [a] * len(n), C.FACTOR_U64, n, timeout_ns=60_000_000_000)
    assert np.all(rep["status"] == C.REPLY_OK)
    assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q)


def _is_prime(n: int) -> bool:
    """Miller-Rabin with the first 12 primes as bases: exact below 3.3e24."""
    if n < 2:
        return False
    bases = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for b in bases:
        if n % b == 0:
            return n == b
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for b in bases:
        x = pow(b, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def test_primes_squares_and_mixed_sizes_split(rt_split):
    """Primes near 2^61 sweep every segment to the bound (about 35,000 tiles)
    and get no divisor; squares of 30-bit primes; small, even and semiprime
    numbers share the batches."""
    rt, a = rt_split
    primes61 = []
    x = (1 << 61) + 10_001
    while len(primes61) < 3:
        if _is_prime(x):
            primes61.append(x)
        x += 2
    p30 = W.primes_uniform(W.stream_key(4243, 1), 3, 1 << 30, 1 << 31)
    squares = [int(v) * int(v) for v in p30]
    n_semi, p_semi, q_semi = W.semiprimes(W.primes_uniform(W.stream_key(4244, 1), 6, 1 << 29, 1 << 31))
    small = [0, 1, 2, 3, 4, 9, 15, 49, 97, 1 << 20, 999_983 * 1_000_003]
    n = np.array(primes61 + squares + [int(v) for v in n_semi] + small, dtype=np.uint64)
    rep = host_requests(rt, [a] * len(n), C.FACTOR_U64, n, timeout_ns=60_000_000_000)
    st, r0, r1 = oracle.factor_batch(np.array(small, dtype=np.uint64))
    want = ([(1, 1, v) for v in primes61] + [(0, int(v), int(v)) for v in p30] +
            [(0, int(pp), int(qq)) for pp, qq in zip(p_semi, q_semi)] +
            [(int(s_), int(a_), int(b_)) for s_, a_, b_ in zip(st, r0, r1)])
    got = [(int(s_), int(a_), int(b_)) for s_, a_, b_ in zip(rep["status"], rep["r0"], rep["r1"])]
    assert got == want


def test_split_matches_oracle_on_a_batch():
    """A routed batch with factors in [2^22, 2^24) (about 276 tiles per batch)
    against the oracle."""
    wl = W.config2(seed=77, n_actors=8, lo=1 << 22, hi=1 << 24, max_messages=200, mean_len=25.0)
    with C.Runtime(max_factor_n=(1 << 50) - 1, max_actors=8, mailbox_capacity=64, factor_split=8) as rt:
        for _ in range(8):
            rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, wl.actor, C.FACTOR_U64, wl.n, wl.sender, wl.sender_seq)
    st, p, q = oracle.factor_batch(wl.n)
    assert np.array_equal(rep["status"], st) and np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q)


def test_split_setting_checked():
    with pytest.raises(C.CafGpuError) as e:
        C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, factor_split=33)
    assert e.value.code == C.EINVAL


@pytest.mark.parametrize("setting,split", [(0, True), (1, False)])
def test_automatic_split_of_a_small_device_batch(setting, split):
    """factor_split 0 (the default) splits the batches of a device batch that
    is smaller than the drain's teams can take; 1 never splits.  One message
    with factors in [2^30, 2^31): unsplit, one team of 8 warps sweeps it (8
    factor items); split, more segments do.  The reply is exact either way."""
    n, p, q = W.semiprimes(W.primes_uniform(W.stream_key(4245, 1), 2, 1 << 30, 1 << 31))
    with C.Runtime(max_actors=4, factor_split=setting) as rt:
        a = rt.spawn(C.FACTOR_U64)
        rt.stats()
        rep = device_batch(rt, np.array([a - 1], np.uint32), C.FACTOR_U64, n)
        st = rt.stats()
    assert rep["status"][0] == C.REPLY_OK and rep["r0"][0] == p[0] and rep["r1"][0] == q[0]
    if split:
        assert st["factor_items"] > 8
    else:
        assert st["factor_items"] == 8
