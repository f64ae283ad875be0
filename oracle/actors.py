"""Sequential reading of the actor semantics -- TEST INFRASTRUCTURE ONLY.

Mailboxes (Sec. 2 "Related Work" and Sec. 3.2 "Lockfree Mailbox
Algorithm"): a mailbox is a FIFO buffer that many actors may append to and
only its owner reads.  Of the two handling categories the paper describes,
the one used here is the strict one: the handler runs exactly once per
message, in arrival order, and no message is skipped (every compute-actor
message matches its handler).  Delivery order between different senders is
not fixed by the paper, so the checker below compares per (sender,
receiver) pair, never a global order.

Token rings (Sec. 5, "Mixed Operations Under Work Load"): rings of actors
pass a token that starts at 1000 and loses one per hop; an actor that
receives 0 terminates.  Readings taken where the paper is silent:

* the decrement is per hop;
* on receiving 0 an actor terminates and forwards 0 once to its successor
  unless the successor has already terminated, so the 0 travels the ring
  once and every actor terminates;
* the ring master (actor 0) sends one factorization request to its ring's
  worker when it starts and one more for every token value v > 0 it
  receives.

Actor creation (Sec. 5, "Overhead of Actor Creation"): 2^N is computed by
recursive creation; an actor with counter N > 0 spawns two actors with
counter N - 1 and waits for their results, an actor with counter 0 answers
1.  Readings: a parent answers the sum of its children's results and then
terminates; every spawned actor terminates after answering.
"""
from __future__ import annotations

from collections import defaultdict, deque

import numpy as np


def simulate_mailboxes(actor: np.ndarray):
    """Deliver messages 0..M-1 in list order to per-actor FIFOs and let every
    actor handle its FIFO front to back.  Returns {actor: [message index, ...]}
    in handling order."""
    fifo = defaultdict(deque)
    for i, a in enumerate(np.asarray(actor).tolist()):
        fifo[a].append(i)
    handled = {}
    for a, q in fifo.items():
        order = []
        while q:
            order.append(q.popleft())
        handled[a] = order
    return handled


def check_mailbox_log(actor, sender, sender_seq, log_actor, log_msg, log_stamp,
                      strict: bool = False):
    """Check a device handling log against the mailbox rules.

    ``log_*`` hold one row per handled message: the actor that handled it, the
    message index and a stamp that increases with handling order.  Checks
    (i) every message is handled exactly once, (ii) by the actor it was sent
    to, (iii) per (sender, receiver) pair in increasing ``sender_seq``.  With
    ``strict`` (a single producer sending in list order) it also checks that
    each actor handled exactly its FIFO of ``simulate_mailboxes``.
    Returns a list of human-readable violations (empty when all hold).
    """
    actor = np.asarray(actor)
    sender = np.asarray(sender)
    sender_seq = np.asarray(sender_seq)
    la = np.asarray(log_actor).astype(np.int64)
    lm = np.asarray(log_msg).astype(np.int64)
    ls = np.asarray(log_stamp).astype(np.int64)
    errs = []
    M = actor.size
    if lm.size != M:
        errs.append(f"log has {lm.size} rows for {M} messages")
    if lm.size and (lm.min() < 0 or lm.max() >= M):
        errs.append("log names a message index out of range")
        return errs
    counts = np.bincount(lm, minlength=M)
    if np.any(counts != 1):
        bad = np.nonzero(counts != 1)[0][:5].tolist()
        errs.append(f"messages not handled exactly once, e.g. {bad}")
    wrong = np.nonzero(actor[lm] != la)[0]
    if wrong.size:
        errs.append(f"{wrong.size} messages handled by the wrong actor")
    order = np.argsort(ls, kind="stable")
    last = {}
    for r in order.tolist():
        m = lm[r]
        key = (int(sender[m]), int(la[r]))
        s = int(sender_seq[m])
        if key in last and last[key] >= s:
            errs.append(f"FIFO broken for sender {key[0]} -> actor {key[1]}: {last[key]} then {s}")
            break
        last[key] = s
    if strict:
        want = simulate_mailboxes(actor)
        got = defaultdict(list)
        for r in order.tolist():
            got[int(la[r])].append(int(lm[r]))
        for a, seq in want.items():
            if got.get(a, []) != seq:
                errs.append(f"actor {a} handled {got.get(a, [])[:8]}... expected {seq[:8]}...")
                break
    return errs


def simulate_rings(n_rings: int, ring_len: int, token: int, incarnations: int = 1):
    """Run every ring to termination, ``incarnations`` times.

    The mixed benchmark's rings are "re-created 4 times" (Sec. 5, "Mixed
    Operations Under Work Load").  Reading: an incarnation is the ring run to
    termination as below; the master then creates the ring anew (new member
    actors, the master itself kept) and starts it with the same token, until
    ``incarnations`` have run; it terminates after the last.  A master sends
    one factorization request when an incarnation starts and one per token
    v > 0 it receives.

    Returns a list with one dict per ring: ``trace`` is the list of
    (receiver, value) deliveries in order over all incarnations (receiver =
    position in the ring, the master at 0), ``incarnation_starts`` the index
    in ``trace`` where each incarnation begins, ``requests`` the number of
    factorization requests the master sent, ``request_after`` the number of
    deliveries seen before each request.
    """
    rings = []
    for _ in range(n_rings):
        trace = []
        req_after = []
        starts = []
        for _inc in range(incarnations):
            done = [False] * ring_len
            starts.append(len(trace))
            req_after.append(len(trace))          # the master's request at the (re)start
            pending = deque([(1 % ring_len, token)])
            while pending:
                r, v = pending.popleft()
                trace.append((r, v))
                succ = (r + 1) % ring_len
                if v > 0:
                    if r == 0:
                        req_after.append(len(trace))
                    pending.append((succ, v - 1))
                else:
                    done[r] = True
                    if not done[succ]:
                        pending.append((succ, 0))
            assert all(done)
        rings.append({"trace": trace, "requests": len(req_after), "request_after": req_after,
                      "incarnation_starts": starts})
    return rings


def source_streams(sources):
    """The messages the SINK / SOURCE reading of the N:1 mailbox experiment
    (Sec. 5, "Mailbox Performance in N:1 Communication Scenario") sends:
    source s (actor index) asked for c messages to sink t sends values
    (s << 32) | k for k = 0 .. c-1, in k order, with sender s and sender
    sequence k.  ``sources``: [(s, c, t), ...].

    Returns (receiver, sender, sender_seq, value) arrays, one row per message,
    each source's messages contiguous and in k order, and {t: (count, sum)}
    with the sum taken mod 2^64 (the sink's counter width)."""
    rec, snd, seq, val = [], [], [], []
    totals = {}
    for s, c, t in sources:
        for k in range(c):
            v = (s << 32) | k
            rec.append(t)
            snd.append(s)
            seq.append(k)
            val.append(v)
            cnt, tot = totals.get(t, (0, 0))
            totals[t] = (cnt + 1, (tot + v) % (1 << 64))
    return (np.asarray(rec, np.int64), np.asarray(snd, np.int64), np.asarray(seq, np.int64),
            np.asarray(val, np.uint64), totals)


def fork_tree(n: int):
    """Run the recursive-creation computation of 2^n as actors exchanging
    messages, one message at a time in arrival order (Sec. 5, "Overhead of
    Actor Creation").

    The root (counter n) gets one start message.  An actor's start message
    with counter c > 0 spawns two actors and sends each a start message with
    counter c - 1; with c = 0 the actor answers 1 at once.  A result message
    adds its value to the actor's sum; after the second result the actor
    answers the sum.  Answering sends a result message to the parent (the
    root's answer is the computation's result) and terminates the actor.

    Returns {"result", "spawned", "messages", "live_after"}: the root's
    answer, the actors spawned (the root not counted), the messages handled
    (start and result messages, including the root's start) and the spawned
    actors still alive at the end."""
    parent = {0: None}
    pending = {0: 0}
    total = {0: 0}
    queue = deque([(0, "start", n)])
    spawned = messages = 0
    result = None
    next_id = 1

    def answer(a, value):
        nonlocal result
        if parent[a] is None:
            result = value
        else:
            queue.append((parent[a], "result", value))
            del parent[a], pending[a], total[a]

    while queue:
        a, kind, v = queue.popleft()
        messages += 1
        if kind == "start":
            if v == 0:
                answer(a, 1)
                continue
            for _ in range(2):
                c = next_id
                next_id += 1
                parent[c], pending[c], total[c] = a, 0, 0
                spawned += 1
                queue.append((c, "start", v - 1))
            pending[a], total[a] = 2, 0
        else:
            total[a] += v
            pending[a] -= 1
            if pending[a] == 0:
                answer(a, total[a])
    return {"result": result, "spawned": spawned, "messages": messages, "live_after": len(parent) - 1}
