"""Pins for the sequential mailbox and token-ring readings."""
import numpy as np

from oracle import actors
from paper_1505_07368_gb300 import workloads as W


def test_simulate_mailboxes_hand_example():
    actor = np.array([2, 0, 2, 1, 0, 2])
    assert actors.simulate_mailboxes(actor) == {2: [0, 2, 5], 0: [1, 4], 1: [3]}


def _valid_log(actor):
    order = actors.simulate_mailboxes(actor)
    la, lm = [], []
    # interleave actors round robin: a valid global order
    its = {a: iter(v) for a, v in order.items()}
    while its:
        for a in list(its):
            try:
                lm.append(next(its[a]))
                la.append(a)
            except StopIteration:
                del its[a]
    return np.array(la), np.array(lm), np.arange(len(lm))


def test_checker_accepts_valid_and_rejects_planted_errors():
    wl = W.config2(n_actors=16, max_messages=300)
    la, lm, ls = _valid_log(wl.actor)
    args = (wl.actor, wl.sender, wl.sender_seq)
    assert actors.check_mailbox_log(*args, la, lm, ls, strict=True) == []
    # duplicate handling
    lm2 = lm.copy(); lm2[5] = lm2[6]
    assert actors.check_mailbox_log(*args, la, lm2, ls)
    # wrong actor
    la2 = la.copy(); la2[3] = (la2[3] + 1) % 16
    assert actors.check_mailbox_log(*args, la2, lm, ls)
    # swap two messages of the same (sender, actor) pair
    key = {}
    for r, m in enumerate(lm.tolist()):
        k = (int(wl.sender[m]), int(la[r]))
        if k in key:
            ls2 = ls.copy(); ls2[key[k]], ls2[r] = ls2[r], ls2[key[k]]
            assert any("FIFO" in e for e in actors.check_mailbox_log(*args, la, lm, ls2))
            break
        key[k] = r
    # missing row
    assert actors.check_mailbox_log(*args, la[:-1], lm[:-1], ls[:-1])


def test_rings_closed_form():
    L, T = 128, 1000
    rings = actors.simulate_rings(3, L, T)
    for r in rings:
        tr = r["trace"]
        assert len(tr) == T + L                     # 1000 nonzero hops + one lap of 0
        for k in range(T + 1):
            assert tr[k] == ((k + 1) % L, T - k)
        assert [v for _, v in tr].count(0) == L
        assert r["requests"] == W.ring_rounds(L, T) == 8
        # the master's nonzero receipts are the deliveries L, 2L, ..., 7L
        assert r["request_after"] == [0] + [k * L for k in range(1, 8)]


def test_rings_small_by_hand():
    # ring of 3, token 2: deliveries a1:2, a2:1, a0:0, a1:0, a2:0
    r = actors.simulate_rings(1, 3, 2)[0]
    assert r["trace"] == [(1, 2), (2, 1), (0, 0), (1, 0), (2, 0)]
    assert r["requests"] == 1


def test_source_streams_closed_form():
    """Sink totals of the N:1 reading against their closed form: source s
    sending c messages contributes c and c (s << 32) + c (c - 1) / 2."""
    from oracle import actors as A
    srcs = [(3, 5, 0), (7, 1, 0), (9, 2000, 1), (1 << 20, 3, 1)]
    rec, snd, seq, val, totals = A.source_streams(srcs)
    assert rec.size == sum(c for _, c, _ in srcs)
    for t in (0, 1):
        want_c = sum(c for s, c, tt in srcs if tt == t)
        want_s = sum(c * (s << 32) + c * (c - 1) // 2 for s, c, tt in srcs if tt == t) % (1 << 64)
        assert totals[t] == (want_c, want_s)
    # each source's messages in k order, values encode (s, k)
    for s, c, _ in srcs:
        rows = snd == s
        assert list(seq[rows]) == list(range(c))
        assert all(int(v) >> 32 == s and int(v) & 0xFFFFFFFF == k for v, k in zip(val[rows], seq[rows]))


def test_fork_tree_by_hand():
    # n = 1: the root spawns two actors with counter 0; each answers 1; the
    # root handles its start and two results and answers 2
    assert actors.fork_tree(1) == {"result": 2, "spawned": 2, "messages": 5, "live_after": 0}
    assert actors.fork_tree(0) == {"result": 1, "spawned": 0, "messages": 1, "live_after": 0}


def test_fork_tree_closed_form():
    # a full binary tree of depth n: 2^n leaves answer 1 each, so the root answers
    # 2^n; it has 2^(n+1) - 1 nodes (the root is not spawned); each of the
    # 2^n - 1 inner nodes handles 3 messages and each leaf 1
    for n in range(0, 13):
        r = actors.fork_tree(n)
        assert r["result"] == 2 ** n
        assert r["spawned"] == 2 ** (n + 1) - 2
        assert r["messages"] == 3 * (2 ** n - 1) + 2 ** n == 2 ** (n + 2) - 3
        assert r["live_after"] == 0


def test_rings_recreated_closed_form():
    # every incarnation repeats the single-incarnation run; requests add up
    L, T, R = 128, 1000, 4
    one = actors.simulate_rings(1, L, T)[0]
    r = actors.simulate_rings(2, L, T, incarnations=R)[1]
    assert r["incarnation_starts"] == [k * (T + L) for k in range(R)]
    assert len(r["trace"]) == R * (T + L)
    for k in range(R):
        assert r["trace"][k * (T + L):(k + 1) * (T + L)] == one["trace"]
        assert r["trace"][k * (T + L)] == (1, T)      # a fresh ring starts at member 1
    assert r["requests"] == R * one["requests"] == 32
    assert r["request_after"] == [k * (T + L) + x for k in range(R) for x in one["request_after"]]


def test_rings_recreated_small_by_hand():
    # ring of 2, token 1, two incarnations: a1:1, a0:0, a1:0 | a1:1, a0:0, a1:0
    r = actors.simulate_rings(1, 2, 1, incarnations=2)[0]
    assert r["trace"] == [(1, 1), (0, 0), (1, 0)] * 2
    assert r["incarnation_starts"] == [0, 3]
    assert r["requests"] == 2 and r["request_after"] == [0, 3]
