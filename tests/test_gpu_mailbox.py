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


def test_n_to_1_sources_into_one_sink():
    """The N:1 mailbox experiment: 40 SOURCE actors stream into one SINK
    concurrently (counts above 1024 exercise the continuation messages); every
    message is handled exactly once, in k order per source, and the sink's
    totals and the sources' replies match the oracle."""
    counts = [700 + 97 * i for i in range(40)]
    # the slot pool is max_actors x the default capacity (the sink's)
    with C.Runtime(max_factor_n=MAX32, max_actors=64, mailbox_capacity=4096, validation_mode=1) as rt:
        sink = rt.spawn(C.SINK)
        srcs = [rt.spawn(C.SOURCE, next=sink, mailbox_capacity=4) for _ in counts]
        msgs = (C.Msg * len(srcs))()
        for i, c in enumerate(counts):
            msgs[i] = C.Runtime.msg(C.SOURCE, u64=c, tag=i)
        h = rt.request_batch(np.array(srcs, np.uint64), msgs)
        rep = rt.await_batch(h, timeout_ns=60_000_000_000)
        # a source replies once it has sent its last message; the sink may
        # still be handling them: wait until everything sent is handled
        rt.sync()
        count, total = rt.sink_totals(sink)
        log = rt.read_log()
    assert np.all(rep["status"] == 0) and list(rep["r0"]) == counts
    rec, snd, seq, val, totals = A.source_streams([(s - 1, c, sink - 1) for s, c in zip(srcs, counts)])
    assert (count, total) == totals[sink - 1]
    rows = log[log["actor"] == sink - 1]
    assert rows.size == rec.size
    # map each handled sink message to its index in the oracle's stream
    index = {(int(s), int(k)): i for i, (s, k) in enumerate(zip(snd, seq))}
    src = rows["sender"].astype(np.int64) & 0x7FFFFFFF
    msg = np.array([index[(int(s), int(k))] for s, k in zip(src, rows["sender_seq"])])
    assert np.array_equal(rows["value"], val[msg])
    errs = A.check_mailbox_log(rec, snd, seq, rows["actor"], msg, rows["stamp"])
    assert errs == []


def test_n_to_1_totals_without_validation_mode():
    """The N:1 experiment outside validation mode, where a SINK takes up to
    128 messages per round of loads: every message counted exactly once, and
    the sink's totals and the sources' replies match the oracle's."""
    counts = [900 + 131 * i for i in range(40)]
    with C.Runtime(max_factor_n=MAX32, max_actors=64, mailbox_capacity=4096) as rt:
        sink = rt.spawn(C.SINK)
        srcs = [rt.spawn(C.SOURCE, next=sink, mailbox_capacity=4) for _ in counts]
        msgs = (C.Msg * len(srcs))()
        for i, c in enumerate(counts):
            msgs[i] = C.Runtime.msg(C.SOURCE, u64=c, tag=i)
        h = rt.request_batch(np.array(srcs, np.uint64), msgs)
        rep = rt.await_batch(h, timeout_ns=60_000_000_000)
        rt.sync()
        count, total = rt.sink_totals(sink)
    assert np.all(rep["status"] == 0) and list(rep["r0"]) == counts
    _, _, _, _, totals = A.source_streams([(s - 1, c, sink - 1) for s, c in zip(srcs, counts)])
    assert (count, total) == totals[sink - 1]


def test_sink_request_replies_count_in_handling_order():
    """Host requests to a SINK: replies are (position in the sink's handling
    order, value), positions 1..N in FIFO order of one sender."""
    vals = [5, 1 << 40, 3, 7, 11] * 20
    with C.Runtime(max_factor_n=MAX32, max_actors=4) as rt:
        sink = rt.spawn(C.SINK)
        msgs = (C.Msg * len(vals))()
        for i, v in enumerate(vals):
            msgs[i] = C.Runtime.msg(C.SINK, u64=v, tag=i)
        h = rt.request_batch(np.full(len(vals), sink, np.uint64), msgs)
        rep = rt.await_batch(h, timeout_ns=60_000_000_000)
        rt.sync()
        count, total = rt.sink_totals(sink)
        rt.reset_actors()
        rt.stream_sync()
        assert rt.sink_totals(sink) == (0, 0)
    assert list(rep["r0"]) == list(range(1, len(vals) + 1))
    assert list(rep["r1"]) == vals
    assert (count, total) == (len(vals), sum(vals))
