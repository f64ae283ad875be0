"""FORK actors: recursive actor creation on the device (Sec. 5, "Overhead of
Actor Creation") against the oracle's message-by-message simulation.

The root's reply must be (2^n, 2^(n+1) - 2) and the drain must handle exactly
the oracle's messages; a pool that fits one tree must serve repeated trees
(the records are recycled)."""
import ctypes

import numpy as np
import pytest

from oracle import actors as OA
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch, host_requests

pytestmark = pytest.mark.gpu


def _run(rt, root, n):
    h = rt.request(root, C.Runtime.msg(C.FORK, u64=n))
    return rt.await_(h, 20_000_000_000)


def test_results_and_counts_match_oracle():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=1 << 14) as rt:
        root = rt.spawn(C.FORK)
        rt.sync()
        rt.stats()
        for n in range(0, 13):
            want = OA.fork_tree(n)
            st, r0, r1 = _run(rt, root, n)
            rt.sync()
            s = rt.stats()
            assert (st, r0, r1) == (C.REPLY_OK, want["result"], want["spawned"]), n
            assert s["device_spawns"] == want["spawned"], n
            assert s["messages"] == want["messages"], n
            assert s["error_word"] == 0


def test_pool_records_are_recycled():
    """A pool of 2046 records holds exactly one n = 10 tree: four trees in a row
    need every record of the previous tree back."""
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=2046) as rt:
        root = rt.spawn(C.FORK)
        rt.sync()
        rt.stats()
        for _ in range(4):
            assert _run(rt, root, 10) == (C.REPLY_OK, 1024, 2046)
        rt.sync()
        assert rt.stats()["device_spawns"] == 4 * 2046
        # the next size up does not fit this pool
        rc = rt.L.caf_gpu_request(rt.h, root, ctypes.byref(C.Runtime.msg(C.FORK, u64=11)),
                                  ctypes.byref(ctypes.c_uint64()))
        assert rc == C.EINVAL


def test_concurrent_roots_share_the_pool():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8, fork_pool=1 << 12) as rt:
        roots = [rt.spawn(C.FORK) for _ in range(4)]
        # 4 trees of n = 9 (1022 records each) fit 4096 records together
        rep = host_requests(rt, roots, C.FORK, [9] * 4, timeout_ns=20_000_000_000)
        assert np.all(rep["status"] == C.REPLY_OK)
        assert np.all(rep["r0"] == 512) and np.all(rep["r1"] == 1022)


def test_device_batch_checks_and_busy_root():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=1 << 17) as rt:
        root = rt.spawn(C.FORK)
        rt.sync()
        # n = 16 is accepted; a second start in the same batch reaches a root
        # that waits for results and is rejected; n = 17 does not fit the pool
        # (2^18 - 2 > 2^17) and n = 31 is out of range
        rep = device_batch(rt, root - 1, C.FORK, [16, 16, 17, 31])
        assert (rep["status"][0], rep["r0"][0], rep["r1"][0]) == (C.REPLY_OK, 1 << 16, (1 << 17) - 2)
        assert list(rep["status"][1:]) == [C.REPLY_REJECTED] * 3
        assert np.all(rep["done"] == 1)
        # the root is ready again afterwards
        assert _run(rt, root, 5) == (C.REPLY_OK, 32, 62)


def test_host_checks():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=1 << 10) as rt:
        root = rt.spawn(C.FORK)
        for n in (10, 31, 1 << 40):    # 2^11 - 2 > 1024; out of range
            rc = rt.L.caf_gpu_request(rt.h, root, ctypes.byref(C.Runtime.msg(C.FORK, u64=n)),
                                      ctypes.byref(ctypes.c_uint64()))
            assert rc == C.EINVAL, n
        assert _run(rt, root, 9) == (C.REPLY_OK, 512, 1022)
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        rc = rt.L.caf_gpu_request(rt.h, root, ctypes.byref(C.Runtime.msg(C.FORK, u64=3)),
                                  ctypes.byref(ctypes.c_uint64()))
        assert rc == C.EINVAL


def test_graph_before_first_fork_spawn_is_refused():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=1 << 10) as rt:
        f = rt.spawn(C.FACTOR_U64)
        rt.graph_begin()
        rt.mark()
        g = rt.graph_end()
        out = ctypes.c_uint64()
        assert rt.L.caf_gpu_spawn(rt.h, C.FORK, None, ctypes.byref(out)) == C.ESTATE
        rt.graph_destroy(g)
        assert f


def test_fork_trees_next_to_factor_actors():
    with C.Runtime(max_factor_n=(1 << 56) - 1, max_actors=8, fork_pool=1 << 15) as rt:
        root = rt.spawn(C.FORK)
        fa = rt.spawn(C.FACTOR_U64)
        nums, p, q = W.semiprimes(W.primes_uniform(W.stream_key(91, 1), 256, 1 << 24, 1 << 28))
        h = rt.request(root, C.Runtime.msg(C.FORK, u64=14))
        fac = host_requests(rt, [fa] * len(nums), C.FACTOR_U64, nums, timeout_ns=20_000_000_000)
        assert rt.await_(h, 20_000_000_000) == (C.REPLY_OK, 1 << 14, (1 << 15) - 2)
        assert np.array_equal(fac["r0"], p) and np.array_equal(fac["r1"], q)
