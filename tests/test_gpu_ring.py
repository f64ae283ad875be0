"""Token rings with factorization workers (the mixed workload) against the
sequential ring reading of the oracle."""
import numpy as np
import pytest

import oracle
from oracle import actors as A
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch, d2h, to_device

pytestmark = pytest.mark.gpu


def build_rings(rt, wl):
    """Spawn per ring: its worker, then actors 0..L-1 (actor 0 is the master)."""
    import torch
    R, L = wl.n_rings, wl.ring_len
    rounds = wl.n.shape[1]
    d_n = to_device(wl.n.astype(np.uint64))
    d_rep = torch.zeros(R * rounds * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    masters, members = [], []
    for r in range(R):
        worker = rt.spawn(C.FACTOR_U64, mailbox_capacity=16)
        base = worker + 1
        ring = []
        for i in range(L):
            nxt = base + (i + 1) % L
            if i == 0:
                h = rt.spawn(C.RING_TOKEN, mailbox_capacity=4, next=nxt, flags=C.ACTOR_MASTER,
                             worker=worker, factor_n=d_n.data_ptr() + r * rounds * 8, factor_count=rounds,
                             factor_replies=d_rep.data_ptr() + r * rounds * C.DREPLY_DTYPE.itemsize)
            else:
                h = rt.spawn(C.RING_TOKEN, mailbox_capacity=4, next=nxt)
            assert h == base + i
            ring.append(h)
        masters.append(ring[0])
        members.append(ring)
    return masters, members, d_n, d_rep


def _check_traces(log, members, wl):
    pos = {}
    for r, ring in enumerate(members):
        for i, h in enumerate(ring):
            pos[h - 1] = (r, i)
    tok = log[((log["kind"] & 0xFFFF) == C.RING_TOKEN) & ((log["kind"] >> 16) & C.MSG_START == 0)]
    tok = tok[np.argsort(tok["stamp"])]
    got = [[] for _ in members]
    for row in tok:
        r, i = pos[int(row["actor"])]
        got[r].append((i, int(row["value"])))
    want = A.simulate_rings(wl.n_rings, wl.ring_len, wl.token)
    for r in range(wl.n_rings):
        assert got[r] == want[r]["trace"], f"ring {r}"


def _check_factors(d_rep, wl):
    rep = d_rep.cpu().numpy().view(C.DREPLY_DTYPE).reshape(wl.n.shape)
    assert np.all(rep["done"] == 1)
    assert np.array_equal(rep["r0"], wl.p) and np.array_equal(rep["r1"], wl.q)
    for x in range(0, wl.n.size, 97):
        r, k = divmod(x, wl.n.shape[1])
        assert oracle.check_certificate(int(wl.n[r, k]), int(rep["r0"][r, k]), int(rep["r1"][r, k]), 0)


def _start(rt, masters, wl):
    idx = np.array([m - 1 for m in masters], np.uint32)
    kind = np.uint32(C.RING_TOKEN | (C.MSG_START << 16))
    return device_batch(rt, idx, kind, np.full(len(masters), wl.token, np.uint64))


@pytest.mark.parametrize("rings,length,token", [(3, 5, 17), (8, 16, 100), (2, 128, 1000)])
def test_small_rings_exact_trace(rings, length, token):
    wl = W.config4(n_rings=rings, ring_len=length, token=token, lo=1 << 14, hi=1 << 16)
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=rings * (length + 1), validation_mode=1) as rt:
        masters, members, d_n, d_rep = build_rings(rt, wl)
        _start(rt, masters, wl)
        log = rt.read_log()
        for ring in members:
            for h in ring:
                assert rt.actor_state(h)[0] == 3
    _check_traces(log, members, wl)
    _check_factors(d_rep, wl)


def test_config4_full_size():
    wl = W.config4()
    with C.Runtime(max_actors=wl.n_rings * (wl.ring_len + 1), validation_mode=1) as rt:
        masters, members, d_n, d_rep = build_rings(rt, wl)
        _start(rt, masters, wl)
        log = rt.read_log()
        # replay after a reset: same traces again
        rt.reset_actors()
        d_rep.zero_()
        _start(rt, masters, wl)
        log2 = rt.read_log()
    _check_traces(log, members, wl)
    _check_traces(log2, members, wl)
    _check_factors(d_rep, wl)


def test_rings_per_message_launch():
    wl = W.config4(n_rings=4, ring_len=8, token=40, lo=1 << 14, hi=1 << 16)
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=64) as rt:
        masters, members, d_n, d_rep = build_rings(rt, wl)
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        for m in masters:
            rt.send(m, C.Runtime.msg(C.RING_TOKEN, wl.token, flags=C.MSG_START))
        rt.sync()
        for ring in members:
            for h in ring:
                assert rt.actor_state(h)[0] == 3
    _check_factors(d_rep, wl)


def test_config4_captured_graph_replays():
    """The whole ring workload (reset the rings, start every master, drain) is
    recorded once as a CUDA graph and replayed; each replay must reproduce the
    exact per-ring traces and the factor replies."""
    import torch
    wl = W.config4()
    with C.Runtime(max_actors=wl.n_rings * (wl.ring_len + 1), validation_mode=1) as rt:
        masters, members, d_n, d_rep = build_rings(rt, wl)
        m = np.zeros(len(masters), C.DMSG_DTYPE)
        m["actor"] = np.array([h - 1 for h in masters], np.uint32)
        m["kind"] = C.RING_TOKEN | (C.MSG_START << 16)
        m["u64"] = wl.token
        d_m = to_device(m)
        d_r = torch.zeros(len(masters) * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        rt.graph_begin()
        rt.reset_actors()
        rt.request_batch_device(d_m.data_ptr(), len(masters), d_r.data_ptr())
        with pytest.raises(C.CafGpuError) as e:
            rt.sync()                         # waiting calls are refused while recording
        assert e.value.code == C.ESTATE
        g = rt.graph_end()
        try:
            for _ in range(3):
                d_rep.zero_()
                torch.cuda.synchronize()
                rt.graph_launch(g)
                rt.stream_sync()
                log = rt.read_log()
                _check_traces(log, members, wl)
                _check_factors(d_rep, wl)
        finally:
            rt.graph_destroy(g)
