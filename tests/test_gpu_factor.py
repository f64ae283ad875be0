"""Parity of the factorization actors with the CPU oracle (bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import d2h, device_batch, host_requests

pytestmark = pytest.mark.gpu

MAX40 = (1 << 40) - 1


def _assert_same(rep, n):
    st, p, q = oracle.factor_batch(np.asarray(n, dtype=np.uint64))
    assert np.array_equal(rep["status"], st), (rep["status"][:8], st[:8])
    assert np.array_equal(rep["r0"], p)
    assert np.array_equal(rep["r1"], q)


def test_prime_table_against_oracle():
    with C.Runtime(max_factor_n=MAX40, max_actors=4) as rt:
        ptr, count = rt.prime_table()
        # odd primes up to 2^20: pi(2^20) = 82025, minus the prime 2
        assert count == 82025 - 1
        host = d2h(ptr, count * 4).view(np.uint32)
    assert host[0] == 3 and host[-1] == 1048573
    assert np.all(np.diff(host.astype(np.int64)) > 0)
    for x in host[::997]:
        assert oracle.is_prime(int(x))


def test_config1_persistent_host_requests():
    wl = W.config1()
    with C.Runtime(max_factor_n=MAX40, max_actors=4, mailbox_capacity=256) as rt:
        a = rt.spawn(C.FACTOR_U64)
        rep = host_requests(rt, np.full(wl.count, a), C.FACTOR_U64, wl.n)
        assert rt.stats()["error_word"] == 0
    _assert_same(rep, wl.n)
    assert np.array_equal(rep["r0"], wl.p) and np.array_equal(rep["r1"], wl.q)


def test_config1_per_message_launch():
    wl = W.config1()
    with C.Runtime(max_factor_n=MAX40, max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        rep = host_requests(rt, np.full(wl.count, a), C.FACTOR_U64, wl.n)
        s = rt.stats()
        assert s["launches"] >= wl.count
    _assert_same(rep, wl.n)


@pytest.mark.parametrize("k,w", [(16, 8), (8, 1), (16, 1), (3, 4), (1, 2), (5, 8), (16, 2)])
def test_config1_device_batch_batching_shapes(k, w):
    wl = W.config1()
    with C.Runtime(max_factor_n=MAX40, max_actors=8, factor_batch=k, factor_warps=w) as rt:
        acts = [rt.spawn(C.FACTOR_U64) for _ in range(5)]
        idx = (np.arange(wl.count) % 5).astype(np.uint32) + np.uint32(acts[0] - 1)
        rep = device_batch(rt, idx, C.FACTOR_U64, wl.n)
        assert np.all(rep["done"] == 1)
    _assert_same(rep, wl.n)


EDGE = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 15, 25, 49, 121, 2 * 3, 97 * 97, 1 << 39, (1 << 40) - 1,
        1048573 * 1048573, 1048573 * 1048571, 1048573, 999983 * 2, 3 * 1048573,
        (1 << 40) - 87]   # last: a prime below 2^40


@pytest.mark.parametrize("backend", [C.BACKEND_PERSISTENT, C.BACKEND_PER_MESSAGE_LAUNCH])
def test_edge_cases(backend):
    n = np.array(EDGE, dtype=np.uint64)
    with C.Runtime(max_factor_n=MAX40, max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        rt.set_backend(backend)
        rep = host_requests(rt, np.full(n.size, a), C.FACTOR_U64, n)
    _assert_same(rep, n)


def test_out_of_range_rejected():
    with C.Runtime(max_factor_n=MAX40, max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        with pytest.raises(C.CafGpuError) as e:
            rt.request(a, C.Runtime.msg(C.FACTOR_U64, 1 << 40))
        assert e.value.code == C.EINVAL
        rep = device_batch(rt, np.array([a - 1, a - 1, a + 5], np.uint32), C.FACTOR_U64,
                           np.array([1 << 40, 35, 35], np.uint64))
        assert rep["status"].tolist() == [C.REPLY_REJECTED, C.REPLY_OK, C.REPLY_REJECTED]
        assert (rep["r0"][1], rep["r1"][1]) == (5, 7)


def test_largest_inputs_full_table():
    """n near 2^62 with the full prime table (odd primes below 2^31)."""
    big_p = 2147483647          # 2^31 - 1, prime
    big_q = 2147483629          # prime
    n = np.array([big_p * big_q, big_q * big_q, (1 << 62) - 1, big_p * 3, big_p], dtype=np.uint64)
    with C.Runtime(max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, np.full(n.size, a - 1, np.uint32), C.FACTOR_U64, n)
    assert (rep["r0"][0], rep["r1"][0]) == (big_q, big_p)
    assert (rep["r0"][1], rep["r1"][1]) == (big_q, big_q)
    assert rep["status"][2] == 0 and int(rep["r0"][2]) * int(rep["r1"][2]) == (1 << 62) - 1
    assert (rep["r0"][2], rep["r1"][2]) == (3, ((1 << 62) - 1) // 3)
    assert (rep["r0"][3], rep["r1"][3]) == (3, big_p)
    assert (rep["status"][4], rep["r0"][4], rep["r1"][4]) == (C.REPLY_NOFACTOR, 1, big_p)


def test_config2_subsample_certificates():
    """1024 actors, factors in [2^24, 2^28): certificate check on every reply, the
    oracle's own trial division on a seeded subsample."""
    wl = W.config2(max_messages=6000)
    with C.Runtime(max_factor_n=(1 << 56) - 1, max_actors=1024, mailbox_capacity=64) as rt:
        for _ in range(wl.n_actors):
            rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, wl.actor, C.FACTOR_U64, wl.n, wl.sender, wl.sender_seq)
    assert np.all(rep["status"] == 0)
    assert np.array_equal(rep["r0"], wl.p) and np.array_equal(rep["r1"], wl.q)
    for i in range(0, wl.count, 499):
        assert oracle.check_certificate(int(wl.n[i]), int(rep["r0"][i]), int(rep["r1"][i]), 0)
    sub = np.arange(0, wl.count, 1500)
    _assert_same(rep[sub], wl.n[sub])


@pytest.mark.parametrize("ingress", ["live", "device"])
def test_grouped_claims_with_small_mailboxes(ingress):
    """Claims that group several batches and sort them by n, with 16-slot mailboxes
    and more messages per actor than a mailbox holds (a claim takes at most one
    mailbox's worth), duplicate n values (ties), primes and even numbers."""
    n_act, per = 384, 40
    _, p, q = W.semiprimes(W.primes_loguniform(W.stream_key(97, 2), 2 * n_act * per, 1 << 10, 1 << 20))
    n = (p.astype(np.uint64) * q.astype(np.uint64))[: n_act * per].copy()
    d = n[3::7].size
    n[0:7 * d:7] = n[3::7]               # duplicates: equal keys in one claim
    n[5::11] = W.primes_uniform(W.stream_key(97, 3), n[5::11].size, 1 << 20, 1 << 30)
    n[9::13] = 2 * (n[9::13] // 2 + 1)
    actors = np.arange(n.size, dtype=np.int64) % n_act
    with C.Runtime(max_factor_n=MAX40, max_actors=n_act, mailbox_capacity=16) as rt:
        ids = [rt.spawn(C.FACTOR_U64) for _ in range(n_act)]
        if ingress == "live":
            rep = host_requests(rt, np.asarray(ids, dtype=np.uint64)[actors], C.FACTOR_U64, n)
        else:
            rep = device_batch(rt, actors.astype(np.uint32), C.FACTOR_U64, n)
        assert rt.stats()["error_word"] == 0
    _assert_same(rep, n)
