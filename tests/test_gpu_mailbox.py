"""Mailbox semantics on the GPU: exactly-once handling, per (sender, receiver)
FIFO order, reply routing, wrap-around and back-pressure, error paths."""
import threading

import numpy as np
import pytest

import oracle
from oracle import actors as A
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch, host_requests

pytestmark = pytest.mark.gpu

MAX32 = (1 << 32) - 1


def _small_factor_workload(n_actors, count, seed=7):
    wl = W.config2(seed=seed, n_actors=n_actors, lo=1 << 12, hi=1 << 16, max_messages=count,
                   mean_len=max(64.0, 2.0 * count / n_actors))
    assert wl.count == count
    return wl


def test_device_batch_strict_fifo_with_wraparound():
    wl = _small_factor_workload(64, 3000)
    with C.Runtime(max_factor_n=MAX32, max_actors=64, mailbox_capacity=8, validation_mode=1,
                   factor_batch=4) as rt:
        for _ in range(64):
            rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, wl.actor, C.FACTOR_U64, wl.n, wl.sender, wl.sender_seq)
        log = rt.read_log()
    errs = A.check_mailbox_log(wl.actor, wl.sender, wl.sender_seq, log["actor"], log["tag"],
                               log["stamp"], strict=True)
    assert errs == []
    assert np.array_equal(log["value"][np.argsort(log["tag"])], wl.n)
    st, p, q = oracle.factor_batch(wl.n)
    assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q) and np.array_equal(rep["status"], st)


def test_host_threads_fifo_per_sender_and_routing():
    n_threads, per_thread, n_actors = 4, 300, 16
    wl = _small_factor_workload(n_actors, n_threads * per_thread, seed=11)
    results = {}
    with C.Runtime(max_factor_n=MAX32, max_actors=n_actors, mailbox_capacity=16, ingress_capacity=64,
                   validation_mode=1) as rt:
        ids = [rt.spawn(C.FACTOR_U64) for _ in range(n_actors)]

        def worker(t):
            out = []
            for i in range(per_thread):
                j = t * per_thread + i
                h = rt.request(ids[int(wl.actor[j])], C.Runtime.msg(C.FACTOR_U64, int(wl.n[j]), sender=t,
                                                                   tag=(t << 32) | i))
                out.append((j, h))
            results[t] = [(j, rt.await_(h, 60_000_000_000)) for j, h in out]

        th = [threading.Thread(target=worker, args=(t,)) for t in range(n_threads)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        rt.sync()
        log = rt.read_log()
    assert log.size == n_threads * per_thread
    # replies routed to the request that asked
    for t in range(n_threads):
        for j, (st, r0, r1) in results[t]:
            assert (st, r0, r1) == oracle.factor(int(wl.n[j]))
    # per (sender, actor): handled in send order
    order = np.argsort(log["stamp"])
    last = {}
    for r in order:
        key = (int(log["sender"][r]), int(log["actor"][r]))
        tag = int(log["tag"][r])
        assert key not in last or last[key] < tag
        last[key] = tag
    assert len(set(log["tag"].tolist())) == log.size


def test_backpressure_single_actor_tiny_mailbox():
    n = np.array([(1 << 31) - 1] * 10 + [35] * 190, dtype=np.uint64)  # mixes slow and fast
    with C.Runtime(max_factor_n=(1 << 62) - 1, max_actors=2, mailbox_capacity=2) as rt:
        a = rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, np.full(n.size, a - 1, np.uint32), C.FACTOR_U64, n)
    st, p, q = oracle.factor_batch(n)
    assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q)


def test_error_paths():
    with C.Runtime(max_factor_n=(1 << 62) - 1, max_actors=8) as rt:
        a = rt.spawn(C.FACTOR_U64)
        with pytest.raises(C.CafGpuError) as e:
            rt.request(a, C.Runtime.msg(C.RING_TOKEN, 5))          # wrong kind for the actor
        assert e.value.code == C.EINVAL
        with pytest.raises(C.CafGpuError) as e:
            rt.request(a + 7, C.Runtime.msg(C.FACTOR_U64, 5))      # no such actor
        assert e.value.code == C.EINVAL
        h = rt.request(a, C.Runtime.msg(C.FACTOR_U64, 91))
        assert rt.await_(h) == (0, 7, 13)
        rc, _ = rt.try_await(h)                                     # already consumed
        assert rc == C.ESTATE
        # a slow request: the smallest factor is close to 2^31
        slow = 2147483629 * 2147483647
        h = rt.request(a, C.Runtime.msg(C.FACTOR_U64, slow))
        rc, _ = rt.try_await(h, timeout_ns=1000)
        assert rc in (C.ETIMEDOUT, C.OK)
        if rc == C.ETIMEDOUT:
            assert rt.await_(h) == (0, 2147483629, 2147483647)


def test_dead_actor_rejects():
    with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=8) as rt:
        a0 = rt.spawn(C.RING_TOKEN, next=2)
        a1 = rt.spawn(C.RING_TOKEN, next=1)
        rt.send(a0, C.Runtime.msg(C.RING_TOKEN, 0))       # token 0: both terminate
        rt.sync()
        assert rt.actor_state(a0)[0] == 3 and rt.actor_state(a1)[0] == 3
        with pytest.raises(C.CafGpuError) as e:
            rt.send(a1, C.Runtime.msg(C.RING_TOKEN, 3))
        assert e.value.code == C.EDEAD


def test_bounded_wait_expiry_reports_and_recovers():
    with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        assert rt.debug_wait_expiry(2_000_000) == C.EWAITLIMIT
        rt.clear_error()
        h = rt.request(a, C.Runtime.msg(C.FACTOR_U64, 1000003 * 999983))
        assert rt.await_(h) == (0, 999983, 1000003)
