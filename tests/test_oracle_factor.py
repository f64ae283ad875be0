"""Pins for the oracle's trial division, independent of the oracle itself."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import workloads as W


def _spf_sieve(limit):
    """Smallest prime factor for every n < limit by the sieve of Eratosthenes."""
    spf = np.zeros(limit, dtype=np.int64)
    for i in range(2, limit):
        if spf[i] == 0:
            spf[i] = i
            if i * i < limit:
                block = spf[i * i::i]
                block[block == 0] = i
    return spf


def test_brute_force_every_n_below_2_20():
    limit = 1 << 20
    spf = _spf_sieve(limit)
    n = np.arange(limit, dtype=np.uint64)
    st, p, q = oracle.factor_batch(n)
    nn = np.arange(limit, dtype=np.int64)
    composite = (nn >= 4) & (spf != nn)
    assert np.array_equal(st == 0, composite)
    assert np.array_equal(p[composite].astype(np.int64), spf[composite])
    assert np.array_equal((p * q)[composite], n[composite])
    # no factor: reply (1, n)
    assert np.all(p[~composite] == 1) and np.array_equal(q[~composite], n[~composite])


@pytest.mark.parametrize("n,expect", [
    (0, (1, 1, 0)), (1, (1, 1, 1)), (2, (1, 1, 2)), (3, (1, 1, 3)),
    (4, (0, 2, 2)), (6, (0, 2, 3)), (9, (0, 3, 3)), (25, (0, 5, 5)),
    (1000003 * 1000003, (0, 1000003, 1000003)),
    (1000003, (1, 1, 1000003)),
    (2 * 2147483647, (0, 2, 2147483647)),
])
def test_special_cases(n, expect):
    assert oracle.factor(n) == expect


def test_matches_generator_certificates_config1():
    wl = W.config1()
    st, p, q = oracle.factor_batch(wl.n)
    assert np.all(st == 0)
    assert np.array_equal(p, wl.p) and np.array_equal(q, wl.q)
    for i in range(0, wl.count, 17):
        assert oracle.check_certificate(int(wl.n[i]), int(p[i]), int(q[i]), 0)


def test_against_sympy_factorint():
    sympy = pytest.importorskip("sympy")
    k = W.stream_key(99, 1)
    xs = W.u64(k, 0, 300) >> np.uint64(24)       # up to 2^40
    st, p, q = oracle.factor_batch(xs)
    for x, s, a, b in zip(xs.tolist(), st.tolist(), p.tolist(), q.tolist()):
        f = sympy.factorint(x)
        if x < 4 or sympy.isprime(x):
            assert (s, a, b) == (1, 1, x)
        else:
            assert s == 0 and a == min(f) and a * b == x


def test_certificate_rejects_wrong_replies():
    n = 1000003 * 999983
    assert oracle.check_certificate(n, 999983, 1000003, 0)
    assert not oracle.check_certificate(n, 1000003, 999983, 0)      # unsorted
    assert not oracle.check_certificate(n + 2, 999983, 1000003, 0)  # product
    assert not oracle.check_certificate(15 * 7, 7, 15, 0)           # 15 not prime
    assert oracle.check_certificate(13, 1, 13, 1)


def test_is_prime_matches_generator_primality():
    xs = np.arange(0, 5000, dtype=np.uint64)
    want = W.is_prime_u32(xs)
    got = np.array([oracle.is_prime(int(x)) for x in xs])
    assert np.array_equal(want, got)
