"""The work-stealing scheduler (a ready queue per CTA, idle CTAs steal; Sec.
6.2) gives the same results as the global ready queue: exactly-once, per
(sender, receiver) FIFO handling, bit-exact factors, the token rings' exact
traces, and the actor-creation tree."""
import numpy as np
import pytest

import oracle
from oracle import actors as A
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch, host_requests

pytestmark = pytest.mark.gpu

MAX32 = (1 << 32) - 1


def test_fifo_and_factors_with_stealing():
    wl = W.config2(seed=17, n_actors=64, lo=1 << 12, hi=1 << 16, max_messages=3000, mean_len=94.0)
    with C.Runtime(max_factor_n=MAX32, max_actors=64, mailbox_capacity=8, validation_mode=1, factor_batch=4,
                   scheduler=C.SCHED_STEAL) as rt:
        for _ in range(64):
            rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, wl.actor, C.FACTOR_U64, wl.n, wl.sender, wl.sender_seq)
        log = rt.read_log()
    errs = A.check_mailbox_log(wl.actor, wl.sender, wl.sender_seq, log["actor"], log["tag"], log["stamp"],
                               strict=True)
    assert errs == []
    st, p, q = oracle.factor_batch(wl.n)
    assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q) and np.array_equal(rep["status"], st)


def test_host_requests_with_stealing():
    wl = W.config2(seed=18, n_actors=256, lo=1 << 16, hi=1 << 20, max_messages=5000, mean_len=40.0)
    with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=256, mailbox_capacity=64,
                   scheduler=C.SCHED_STEAL) as rt:
        actors = [rt.spawn(C.FACTOR_U64) for _ in range(256)]
        rep = host_requests(rt, np.array(actors, np.uint64)[wl.actor], C.FACTOR_U64, wl.n,
                            timeout_ns=20_000_000_000)
    st, p, q = oracle.factor_batch(wl.n)
    assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q) and np.array_equal(rep["status"], st)


def test_fork_tree_with_stealing():
    with C.Runtime(max_factor_n=MAX32, max_actors=4, fork_pool=1 << 15, scheduler=C.SCHED_STEAL) as rt:
        root = rt.spawn(C.FORK)
        rt.sync()
        rt.stats()
        for n in (0, 1, 5, 10, 14):
            want = A.fork_tree(n)
            h = rt.request(root, C.Runtime.msg(C.FORK, u64=n))
            assert rt.await_(h, 20_000_000_000) == (C.REPLY_OK, want["result"], want["spawned"]), n
            rt.sync()
            s = rt.stats()
            assert s["device_spawns"] == want["spawned"] and s["messages"] == want["messages"], n


def test_invalid_scheduler_rejected():
    with pytest.raises(C.CafGpuError) as e:
        C.Runtime(max_factor_n=MAX32, max_actors=4, scheduler=2)
    assert e.value.code == C.EINVAL
