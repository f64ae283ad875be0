"""Token rings whose master re-creates the ring on the device (the mixed
benchmark's rings "re-created 4 times", Sec. 5) against the oracle's
re-created ring reading: every incarnation's trace, the factorization
requests of all incarnations, the spawn count, and record recycling."""
import numpy as np
import pytest

import oracle
from oracle import actors as A
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch, to_device

pytestmark = pytest.mark.gpu


def _spawn_masters(rt, n_rings, ring_len, incarnations, wl):
    import torch
    rounds = wl.n.shape[1]
    d_n = to_device(wl.n.astype(np.uint64))
    d_rep = torch.zeros(n_rings * rounds * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    masters = []
    for r in range(n_rings):
        worker = rt.spawn(C.FACTOR_U64, mailbox_capacity=16)
        masters.append(rt.spawn(C.RING_TOKEN, mailbox_capacity=4, flags=C.ACTOR_MASTER | C.ACTOR_RECREATE,
                                worker=worker, factor_n=d_n.data_ptr() + r * rounds * 8, factor_count=rounds,
                                factor_replies=d_rep.data_ptr() + r * rounds * C.DREPLY_DTYPE.itemsize,
                                ring_len=ring_len, incarnations=incarnations))
    return masters, d_n, d_rep


def _workload(n_rings, ring_len, token, incarnations):
    one = W.config4(n_rings=n_rings, ring_len=ring_len, token=token, lo=1 << 14, hi=1 << 16)
    wl = W.config4(n_rings=n_rings * incarnations, ring_len=ring_len, token=token, lo=1 << 14, hi=1 << 16)
    rounds = one.n.shape[1] * incarnations
    wl.n = wl.n.reshape(n_rings, rounds)
    wl.p = wl.p.reshape(n_rings, rounds)
    wl.q = wl.q.reshape(n_rings, rounds)
    return wl


def _traces(log, masters):
    """Per master: [(incarnation, position, value)] in handling order, from the
    ring label the tokens carry in their tag."""
    tok = log[((log["kind"] & 0xFFFF) == C.RING_TOKEN) & ((log["kind"] >> 16) == 0)]
    tok = tok[np.argsort(tok["stamp"])]
    idx = {m - 1: r for r, m in enumerate(masters)}
    got = [[] for _ in masters]
    for row in tok:
        tag = int(row["tag"])
        got[idx[(tag & 0xFFFFFFFF) - 1]].append(((tag >> 32) & 0xFF, tag >> 40, int(row["value"]) & 0xFFFFFFFF))
    return got


def _check(log, masters, ring_len, token, incarnations):
    want = A.simulate_rings(len(masters), ring_len, token, incarnations=incarnations)
    for r, got in enumerate(_traces(log, masters)):
        assert [(p, v) for _, p, v in got] == want[r]["trace"], f"ring {r}"
        starts = want[r]["incarnation_starts"] + [len(got)]
        for k in range(incarnations):
            assert all(inc == k for inc, _, _ in got[starts[k]:starts[k + 1]]), (r, k)


@pytest.mark.parametrize("rings,length,token,incs", [(3, 5, 17, 3), (4, 2, 3, 2), (2, 40, 100, 4)])
def test_recreated_rings_exact_trace(rings, length, token, incs):
    wl = _workload(rings, length, token, incs)
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=2 * rings, validation_mode=1,
                   fork_pool=1 << 12) as rt:
        masters, d_n, d_rep = _spawn_masters(rt, rings, length, incs, wl)
        rt.stats()
        rep = device_batch(rt, np.array([m - 1 for m in masters], np.uint32),
                           np.uint32(C.RING_TOKEN | (C.MSG_START << 16)), np.full(rings, token, np.uint64))
        st = rt.stats()
        log = rt.read_log()
        states = [rt.actor_state(m)[0] for m in masters]
    assert np.all(rep["status"] == 0) and np.all(rep["r0"] == token)
    _check(log, masters, length, token, incs)
    assert st["device_spawns"] == rings * (length - 1) * incs
    assert states == [3] * rings                  # every master terminated after its last incarnation
    fr = d_rep.cpu().numpy().view(C.DREPLY_DTYPE).reshape(wl.n.shape)
    n_req = A.simulate_rings(1, length, token, incarnations=incs)[0]["requests"]
    assert np.all(fr["done"][:, :n_req] == 1)
    assert np.array_equal(fr["r0"][:, :n_req], wl.p[:, :n_req]) and np.array_equal(fr["r1"][:, :n_req], wl.q[:, :n_req])


def test_config4_rings_recreated_four_times_with_a_tight_pool():
    """64 rings of 128 actors, token 1000, re-created 4 times, factor requests
    in [2^30, 2^31); the pool holds one incarnation of every ring, so the four
    incarnations run only if terminated members return their records."""
    R, L, T, I = 64, 128, 1000, 4
    base = W.config4()
    wl = W.config4(n_rings=R * I)
    wl.n, wl.p, wl.q = (x.reshape(R, base.n.shape[1] * I) for x in (wl.n, wl.p, wl.q))
    with C.Runtime(max_actors=2 * R, validation_mode=1, fork_pool=R * (L - 1)) as rt:
        masters, d_n, d_rep = _spawn_masters(rt, R, L, I, wl)
        rt.stats()
        rep = device_batch(rt, np.array([m - 1 for m in masters], np.uint32),
                           np.uint32(C.RING_TOKEN | (C.MSG_START << 16)), np.full(R, T, np.uint64))
        st = rt.stats()
        log = rt.read_log()
    assert np.all(rep["status"] == 0)
    _check(log, masters, L, T, I)
    assert st["device_spawns"] == R * (L - 1) * I
    fr = d_rep.cpu().numpy().view(C.DREPLY_DTYPE).reshape(wl.n.shape)
    assert np.all(fr["done"] == 1)
    assert np.array_equal(fr["r0"], wl.p) and np.array_equal(fr["r1"], wl.q)
    for x in range(0, wl.n.size, 101):
        r, k = divmod(x, wl.n.shape[1])
        assert oracle.check_certificate(int(wl.n[r, k]), int(fr["r0"][r, k]), int(fr["r1"][r, k]), 0)


def test_second_start_while_running_is_rejected_and_replay_after_reset():
    wl = _workload(1, 6, 20, 2)
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=2, validation_mode=1, fork_pool=64) as rt:
        masters, d_n, d_rep = _spawn_masters(rt, 1, 6, 2, wl)
        m = masters[0] - 1
        rep = device_batch(rt, np.array([m, m], np.uint32), np.uint32(C.RING_TOKEN | (C.MSG_START << 16)),
                           np.array([20, 20], np.uint64))
        assert list(rep["status"]) == [C.REPLY_OK, C.REPLY_REJECTED]
        rt.read_log()
        # reset and run again: the recycled pool records serve the new rings
        rt.reset_actors()
        rt.stream_sync()
        rep = device_batch(rt, np.array([m], np.uint32), np.uint32(C.RING_TOKEN | (C.MSG_START << 16)),
                           np.array([20], np.uint64))
        assert rep["status"][0] == C.REPLY_OK
        log = rt.read_log()
    _check(log, masters, 6, 20, 2)


def test_recreate_spawn_checks():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4, fork_pool=16) as rt:
        w = rt.spawn(C.FACTOR_U64)
        for bad in ({"ring_len": 1, "incarnations": 1}, {"ring_len": 4, "incarnations": 0},
                    {"ring_len": 4, "incarnations": 256}, {"ring_len": 18, "incarnations": 1}):
            with pytest.raises(C.CafGpuError) as e:
                rt.spawn(C.RING_TOKEN, flags=C.ACTOR_MASTER | C.ACTOR_RECREATE, worker=w, **bad)
            assert e.value.code == C.EINVAL, bad
        with pytest.raises(C.CafGpuError):
            rt.spawn(C.RING_TOKEN, flags=C.ACTOR_RECREATE, worker=w, ring_len=4, incarnations=1)
        a = rt.spawn(C.RING_TOKEN, flags=C.ACTOR_MASTER | C.ACTOR_RECREATE, worker=w, ring_len=4, incarnations=1)
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        with pytest.raises(C.CafGpuError) as e:
            rt.send(a, C.Runtime.msg(C.RING_TOKEN, 5, flags=C.MSG_START))
        assert e.value.code == C.EINVAL
