"""GEMM actors at the serving workload's largest sizes, n in (1024, 2048].

These sizes run through the drain's large scratch class (packed images of up
to 128 MB per message) and up to 16 x 16 output tiles per message.  Operands
are N(0,1) and integer-valued matrices; the float64 oracle is computed on
sampled rows (every 128-row tile's first and last row and a random one, so
every output tile is covered) and, for two integer cases, in full.  Bounds per
size: relative Frobenius error <= 1e-2 (BF16) and <= 1e-5 (split-BF16x3);
integer-valued products are exact.
"""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [1025, 1100, 1536, 2047, 2048]
TOL = {C.GEMM_BF16: 1e-2, C.GEMM_SPLIT_BF16X3: 1e-5}
KINDS = (C.GEMM_BF16, C.GEMM_SPLIT_BF16X3)


def _sample_rows(n: int, seed: int) -> np.ndarray:
    tiles = (n + 127) // 128
    r = W.u64(W.stream_key(seed, n), 0, tiles)
    rows = []
    for t in range(tiles):
        lo, hi = 128 * t, min(128 * t + 127, n - 1)
        rows += [lo, hi, lo + int(r[t] % np.uint64(hi - lo + 1))]
    return np.unique(np.array(rows, np.int64))


def _normal_operands(n: int, seed: int):
    A = W.normal_f32(W.stream_key(seed, 2 * n), 0, n * n).reshape(n, n)
    B = W.normal_f32(W.stream_key(seed, 2 * n + 1), 0, n * n).reshape(n, n)
    return A, B


def _drain_batch(rt, actors, kinds, mats):
    """One device batch: message i multiplies mats[i] = (A, B) on actor actors[i]."""
    import torch
    from helpers import to_device
    count = len(mats)
    dev = [(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()) for A, B in mats]
    outs = [torch.full(A.shape, float("nan"), dtype=torch.float32, device="cuda") for A, _ in mats]
    desc = np.zeros(count, C.GEMM_DESC_DTYPE)
    for i, ((dA, dB), o) in enumerate(zip(dev, outs)):
        desc[i] = (dA.data_ptr(), dB.data_ptr(), o.data_ptr(), o.shape[0], 0)
    d_desc = to_device(desc)
    m = np.zeros(count, C.DMSG_DTYPE)
    m["actor"] = np.asarray(actors, np.uint32) - 1
    m["kind"] = kinds
    m["u64"] = d_desc.data_ptr() + np.arange(count, dtype=np.uint64) * C.GEMM_DESC_DTYPE.itemsize
    m["tag"] = np.arange(count)
    d_m = to_device(m)
    d_r = torch.zeros(count * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rt.request_batch_device(d_m.data_ptr(), count, d_r.data_ptr())
    rt.stream_sync()
    rep = d_r.cpu().numpy().view(C.DREPLY_DTYPE).copy()
    st = rt.stats()
    return rep, [o.cpu().numpy() for o in outs], st


def test_drain_large_sizes_error_per_size():
    """Twenty messages (five sizes x two kinds x two copies) in one drain: more
    than the 16 large scratch records, so records are reused within the batch."""
    ops = {n: _normal_operands(n, 61) for n in SIZES}
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        act = {C.GEMM_BF16: rt.spawn(C.GEMM_BF16), C.GEMM_SPLIT_BF16X3: rt.spawn(C.GEMM_SPLIT_BF16X3)}
        plan = [(n, k) for _ in range(2) for n in SIZES for k in KINDS]
        rep, outs, st = _drain_batch(rt, [act[k] for _, k in plan], np.array([k for _, k in plan], np.uint32),
                                     [ops[n] for n, _ in plan])
    assert np.all(rep["done"] == 1) and np.all(rep["status"] == 0)
    assert np.array_equal(rep["r1"], np.array([n for n, _ in plan], np.uint64))
    assert st["gemm_tiles"] == sum(((n + 127) // 128) ** 2 for n, _ in plan)
    half = len(plan) // 2
    for i in range(half):
        # a tile's arithmetic does not depend on scheduling: both copies agree bit for bit
        assert np.array_equal(outs[i].view(np.uint32), outs[i + half].view(np.uint32)), plan[i]
    print("\nGEMM-ERROR-TABLE-LARGE n kind rows err")
    for i in range(half):
        n, k = plan[i]
        A, B = ops[n]
        rows = _sample_rows(n, 62)
        err = oracle.rel_frobenius(outs[i][rows], oracle.gemm_rows(A, B, rows))
        print(f"GEMM-ERROR-TABLE-LARGE {n} {'bf16' if k == C.GEMM_BF16 else 'split'} {rows.size} {err:.3e}")
        assert err <= TOL[k], (n, k, err)


@pytest.mark.parametrize("n", [1025, 2048])
def test_drain_large_integer_matrices_exact_in_full(n):
    A = W.integer_matrix(W.stream_key(63, n), n)
    B = W.integer_matrix(W.stream_key(64, n), n)
    want = oracle.gemm_f64(A, B)
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        act = [rt.spawn(k) for k in KINDS]
        rep, outs, _ = _drain_batch(rt, act, np.array(KINDS, np.uint32), [(A, B), (A, B)])
    assert np.all(rep["done"] == 1) and np.all(rep["status"] == 0)
    for k, got in zip(KINDS, outs):
        assert np.array_equal(got.astype(np.float64), want), (n, k, np.nanmax(np.abs(got - want)))


def _per_message(rt, actor, kind, A, B):
    import torch
    n = A.shape[0]
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    h = rt.request(actor, C.Runtime.msg(kind, n=n, A=dA.data_ptr(), B=dB.data_ptr(), C=dC.data_ptr()))
    st, _, r1 = rt.await_(h, 120_000_000_000)
    assert (st, r1) == (0, n)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def test_per_message_launch_large_sizes():
    """The per-message-launch comparator at the same sizes: N(0,1) error per
    size on sampled rows, and an integer-valued product exact on them."""
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        act = {k: rt.spawn(k) for k in KINDS}
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        for n in SIZES:
            A, B = _normal_operands(n, 65)
            rows = _sample_rows(n, 66)
            want = oracle.gemm_rows(A, B, rows)
            for k in KINDS:
                err = oracle.rel_frobenius(_per_message(rt, act[k], k, A, B)[rows], want)
                assert err <= TOL[k], (n, k, err)
        n = 2047
        A = W.integer_matrix(W.stream_key(67, n), n)
        B = W.integer_matrix(W.stream_key(68, n), n)
        rows = _sample_rows(n, 69)
        want = oracle.gemm_rows(A, B, rows)
        for k in KINDS:
            assert np.array_equal(_per_message(rt, act[k], k, A, B)[rows].astype(np.float64), want), k


def test_serving_mix_with_large_gemms():
    """Serving with GEMMs up to n = 2048 in the mix (the serving workload's full
    size range): every factorization reply against the generator's factors, and
    every large GEMM (n > 1024) against the oracle on sampled rows."""
    import torch
    wl = W.config5(seed=70, n_requests=400, rate=2e3, factor_hi=1 << 22, pool_elems=1 << 24,
                   n_factor_actors=8, n_gemm_actors=8)
    pool_np = W.gemm_pool(wl.pool_seed, wl.pool_elems)
    pool = torch.from_numpy(pool_np).cuda()
    arena = torch.zeros(2 << 30, dtype=torch.uint8, device="cuda")
    isf = wl.kind == C.FACTOR_U64
    big = np.nonzero(~isf & (wl.size > 1024))[0]
    assert big.size >= 3, big.size          # the draw reaches the large class
    with C.Runtime(max_factor_n=(1 << 44) - 1, max_actors=32, mailbox_capacity=256) as rt:
        fa = [rt.spawn(C.FACTOR_U64, mailbox_capacity=256) for _ in range(8)]
        ga = [rt.spawn(C.GEMM_SPLIT_BF16X3, mailbox_capacity=256) for _ in range(8)]
        reqs = np.zeros(wl.count, C.SERVE_REQ_DTYPE)
        reqs["actor"] = np.where(isf, np.array(fa, np.uint64)[wl.actor % 8], np.array(ga, np.uint64)[wl.actor % 8])
        reqs["t_arrival"] = wl.t
        reqs["u64"] = wl.n
        reqs["n"] = wl.size
        reqs["A"] = np.where(isf, 0, pool.data_ptr() + 4 * wl.a_off.astype(np.uint64))
        reqs["B"] = np.where(isf, 0, pool.data_ptr() + 4 * wl.b_off.astype(np.uint64))
        torch.cuda.synchronize()
        res, st = rt.serve_run(reqs, arena.data_ptr(), arena.numel(), mem_budget_bytes=1 << 30,
                               timeout_ns=120_000_000_000)
    torch.cuda.synchronize()
    assert st["peak_inflight_bytes"] <= 1 << 30
    assert np.all(res["status"] == 0)
    fi = np.nonzero(isf)[0]
    assert np.array_equal(res["r0"][fi], wl.p[fi]) and np.array_equal(res["r1"][fi], wl.q[fi])
    arena_np = arena.cpu().numpy()
    for i in big:
        n = int(wl.size[i])
        A = pool_np[wl.a_off[i]:wl.a_off[i] + n * n].reshape(n, n)
        B = pool_np[wl.b_off[i]:wl.b_off[i] + n * n].reshape(n, n)
        off = int(res["c_offset"][i])
        got = arena_np[off:off + 4 * n * n].view(np.float32).reshape(n, n)
        rows = _sample_rows(n, 71)
        assert oracle.rel_frobenius(got[rows], oracle.gemm_rows(A, B, rows)) <= 1e-5, (i, n)
