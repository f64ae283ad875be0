"""GEMM actors (tcgen05, BF16 and split-BF16x3) against the float64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(rt, actor, kind, A, B, backend=C.BACKEND_PER_MESSAGE_LAUNCH):
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
