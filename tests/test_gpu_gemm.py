"""GEMM actors (tcgen05, BF16 and split-BF16x3) against the float64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(rt, actor, kind, A, B, backend=None):
    import torch
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    h = rt.request(actor, C.Runtime.msg(kind, n=n, A=dA.data_ptr(), B=dB.data_ptr(), C=dC.data_ptr()))
    st, r0, r1 = rt.await_(h, 60_000_000_000)
    assert (st, r1) == (0, n)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.fixture(scope="module")
def rt_pm():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        a_bf16 = rt.spawn(C.GEMM_BF16)
        a_split = rt.spawn(C.GEMM_SPLIT_BF16X3)
        rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        yield rt, a_bf16, a_split


@pytest.mark.parametrize("n", [64, 128, 33, 200, 256, 320])
def test_integer_matrices_exact(rt_pm, n):
    rt, a_bf16, a_split = rt_pm
    A = W.integer_matrix(W.stream_key(21, n), n)
    B = W.integer_matrix(W.stream_key(22, n), n)
    want = oracle.gemm_f64(A, B)
    for actor, kind in ((a_bf16, C.GEMM_BF16), (a_split, C.GEMM_SPLIT_BF16X3)):
        got = _run(rt, actor, kind, A, B)
        assert np.array_equal(got.astype(np.float64), want), (kind, np.nanmax(np.abs(got - want)))


def test_identity_and_transpose_sensitivity(rt_pm):
    rt, a_bf16, a_split = rt_pm
    n = 128
    A = W.integer_matrix(W.stream_key(23, n), n)
    I = np.eye(n, dtype=np.float32)
    assert np.array_equal(_run(rt, a_split, C.GEMM_SPLIT_BF16X3, A, I), A)
    assert np.array_equal(_run(rt, a_split, C.GEMM_SPLIT_BF16X3, I, A), A)
    # A*B differs from B*A and from A^T*B: a transposed operand would show
    B = W.integer_matrix(W.stream_key(24, n), n)
    got = _run(rt, a_bf16, C.GEMM_BF16, A, B)
    assert np.array_equal(got.astype(np.float64), oracle.gemm_f64(A, B))
    assert not np.array_equal(got.astype(np.float64), oracle.gemm_f64(B, A))


@pytest.mark.parametrize("n", [64, 192, 512, 1024])
def test_normal_matrices_error_bounds(rt_pm, n):
    rt, a_bf16, a_split = rt_pm
    A = W.normal_f32(W.stream_key(25, n), 0, n * n).reshape(n, n)
    B = W.normal_f32(W.stream_key(26, n), 0, n * n).reshape(n, n)
    C64 = oracle.gemm_f64(A, B)
    e_bf16 = oracle.rel_frobenius(_run(rt, a_bf16, C.GEMM_BF16, A, B), C64)
    e_split = oracle.rel_frobenius(_run(rt, a_split, C.GEMM_SPLIT_BF16X3, A, B), C64)
    assert e_bf16 <= 1e-2, e_bf16
    assert e_split <= 1e-5, e_split
    assert e_split < e_bf16 / 50


# ---- GEMM actors in the persistent drain -----------------------------------

def test_persistent_host_requests():
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        a_bf16 = rt.spawn(C.GEMM_BF16)
        a_split = rt.spawn(C.GEMM_SPLIT_BF16X3)
        for n in (64, 100, 256):
            A = W.integer_matrix(W.stream_key(31, n), n)
            B = W.integer_matrix(W.stream_key(32, n), n)
            want = oracle.gemm_f64(A, B)
            for actor, kind in ((a_bf16, C.GEMM_BF16), (a_split, C.GEMM_SPLIT_BF16X3)):
                got = _run(rt, actor, kind, A, B, backend=C.BACKEND_PERSISTENT)
                assert np.array_equal(got.astype(np.float64), want), (n, kind)


def _gemm_device_batch(rt, actor_idx, kinds, sizes, pool, seed):
    """Device batch of GEMM messages with operands at seeded offsets in `pool` (device)."""
    import torch
    from helpers import to_device
    count = len(sizes)
    offs_a = W._offsets(W.stream_key(seed, 1), np.asarray(sizes), pool.numel())
    offs_b = W._offsets(W.stream_key(seed, 2), np.asarray(sizes), pool.numel())
    outs = [torch.full((int(n), int(n)), float("nan"), dtype=torch.float32, device="cuda") for n in sizes]
    desc = np.zeros(count, C.GEMM_DESC_DTYPE)
    base = pool.data_ptr()
    for i, n in enumerate(sizes):
        desc[i] = (base + 4 * int(offs_a[i]), base + 4 * int(offs_b[i]), outs[i].data_ptr(), int(n), 0)
    d_desc = to_device(desc)
    m = np.zeros(count, C.DMSG_DTYPE)
    m["actor"] = actor_idx
    m["kind"] = kinds
    m["u64"] = d_desc.data_ptr() + np.arange(count, dtype=np.uint64) * C.GEMM_DESC_DTYPE.itemsize
    m["tag"] = np.arange(count)
    d_m = to_device(m)
    d_r = torch.zeros(count * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rt.request_batch_device(d_m.data_ptr(), count, d_r.data_ptr())
    rt.stream_sync()
    rep = d_r.cpu().numpy().view(C.DREPLY_DTYPE).copy()
    return rep, offs_a, offs_b, [o.cpu().numpy() for o in outs]


def test_persistent_device_batch_mixed_sizes_and_kinds():
    import torch
    pool_np = W.gemm_pool(33, 1 << 21)
    pool = torch.from_numpy(pool_np).cuda()
    sizes = [64, 128, 200, 256, 33, 512, 96, 384, 448, 64, 160, 320]
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        acts = [rt.spawn(C.GEMM_BF16), rt.spawn(C.GEMM_SPLIT_BF16X3), rt.spawn(C.GEMM_SPLIT_BF16X3)]
        idx = np.array([acts[i % 3] - 1 for i in range(len(sizes))], np.uint32)
        kinds = np.array([C.GEMM_BF16 if i % 3 == 0 else C.GEMM_SPLIT_BF16X3 for i in range(len(sizes))], np.uint32)
        rep, oa, ob, outs = _gemm_device_batch(rt, idx, kinds, sizes, pool, 34)
        st = rt.stats()
    assert np.all(rep["done"] == 1) and np.all(rep["status"] == 0)
    assert np.array_equal(rep["r1"], np.array(sizes, np.uint64))
    expected_tiles = sum(((n + 127) // 128) ** 2 for n in sizes)
    assert st["gemm_tiles"] == expected_tiles
    for i, n in enumerate(sizes):
        A = pool_np[oa[i]:oa[i] + n * n].reshape(n, n)
        B = pool_np[ob[i]:ob[i] + n * n].reshape(n, n)
        err = oracle.rel_frobenius(outs[i], oracle.gemm_f64(A, B))
        assert err <= (1e-2 if kinds[i] == C.GEMM_BF16 else 1e-5), (n, kinds[i], err)


def test_persistent_factor_and_gemm_in_one_drain():
    import torch
    pool_np = W.gemm_pool(35, 1 << 20)
    pool = torch.from_numpy(pool_np).cuda()
    wl = W.config1()
    with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=8) as rt:
        f = rt.spawn(C.FACTOR_U64)
        g = rt.spawn(C.GEMM_SPLIT_BF16X3)
        # GEMM batch and factor batch back to back on the runtime stream
        from helpers import device_batch
        sizes = [256, 128, 64, 300]
        rep_g, oa, ob, outs = _gemm_device_batch(rt, np.full(len(sizes), g - 1, np.uint32),
                                                 np.full(len(sizes), C.GEMM_SPLIT_BF16X3, np.uint32), sizes, pool, 36)
        rep_f = device_batch(rt, np.full(wl.count, f - 1, np.uint32), C.FACTOR_U64, wl.n)
    st, p, q = oracle.factor_batch(wl.n)
    assert np.array_equal(rep_f["r0"], p) and np.array_equal(rep_f["r1"], q)
    for i, n in enumerate(sizes):
        A = pool_np[oa[i]:oa[i] + n * n].reshape(n, n)
        B = pool_np[ob[i]:ob[i] + n * n].reshape(n, n)
        assert oracle.rel_frobenius(outs[i], oracle.gemm_f64(A, B)) <= 1e-5


def test_error_table_every_workload_size():
    """Relative Frobenius error against the float64 oracle for every n of the
    GEMM-actor workload (64, 128, ..., 1024), N(0,1) operands, BF16 and split
    forms of the same product, through the persistent drain.  Prints the table."""
    import torch
    from helpers import to_device
    sizes = list(range(64, 1025, 64))
    pool_np = W.gemm_pool(37, 1 << 21)
    pool = torch.from_numpy(pool_np).cuda()
    offs_a = W._offsets(W.stream_key(37, 1), np.asarray(sizes), pool.numel())
    offs_b = W._offsets(W.stream_key(37, 2), np.asarray(sizes), pool.numel())
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4) as rt:
        a_bf, a_sp = rt.spawn(C.GEMM_BF16), rt.spawn(C.GEMM_SPLIT_BF16X3)
        outs = [torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda") for n in sizes for _ in (0, 1)]
        count = len(outs)
        desc = np.zeros(count, C.GEMM_DESC_DTYPE)
        m = np.zeros(count, C.DMSG_DTYPE)
        for i, n in enumerate(sizes):
            for k, (actor, kind) in enumerate(((a_bf, C.GEMM_BF16), (a_sp, C.GEMM_SPLIT_BF16X3))):
                j = 2 * i + k
                desc[j] = (pool.data_ptr() + 4 * int(offs_a[i]), pool.data_ptr() + 4 * int(offs_b[i]),
                           outs[j].data_ptr(), n, 0)
                m[j]["actor"] = actor - 1
                m[j]["kind"] = kind
                m[j]["tag"] = j
        d_desc = to_device(desc)
        m["u64"] = d_desc.data_ptr() + np.arange(count, dtype=np.uint64) * C.GEMM_DESC_DTYPE.itemsize
        d_m = to_device(m)
        d_r = torch.zeros(count * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        rt.request_batch_device(d_m.data_ptr(), count, d_r.data_ptr())
        rt.stream_sync()
        rep = d_r.cpu().numpy().view(C.DREPLY_DTYPE)
        got = [o.cpu().numpy() for o in outs]
    assert np.all(rep["done"] == 1) and np.all(rep["status"] == 0)
    print("\nGEMM-ERROR-TABLE n bf16 split")
    for i, n in enumerate(sizes):
        A = pool_np[offs_a[i]:offs_a[i] + n * n].reshape(n, n)
        B = pool_np[offs_b[i]:offs_b[i] + n * n].reshape(n, n)
        C64 = oracle.gemm_f64(A, B)
        e_bf, e_sp = oracle.rel_frobenius(got[2 * i], C64), oracle.rel_frobenius(got[2 * i + 1], C64)
        print(f"GEMM-ERROR-TABLE {n} {e_bf:.3e} {e_sp:.3e}")
        assert e_bf <= 1e-2, (n, e_bf)
        assert e_sp <= 1e-5, (n, e_sp)
