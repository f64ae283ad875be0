"""caf_gpu_factor_static: the factorization call that allocates no device memory.

It is meant for callers that cannot call cudaMalloc (a host framework whose
allocator owns the GPU's memory, latency-critical paths, programs that forbid
allocation after start-up).  This test calls it through the C ABI, twice in a
row with different numbers (so a stale scratch word from the first call would
show in the second), and requires the same replies as the runtime's device
batch entry point.  The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch

pytestmark = pytest.mark.gpu

MAX40 = (1 << 40) - 1
EDGE = [0, 1, 2, 3, 4, 5, 8, 9, 15, 25, 49, 97 * 97, 1 << 39, MAX40, 1048573 * 1048573,
        1048573 * 1048571, 1048573, 999983 * 2, 3 * 1048573, (1 << 40) - 87]


def _static_call(values: np.ndarray) -> np.ndarray:
    import torch
    d_n = torch.from_numpy(values.astype(np.uint64).view(np.uint8).copy()).cuda()
    d_rep = torch.zeros(values.size * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rc = C.factor_static(d_n.data_ptr(), values.size, d_rep.data_ptr(), 0)
    assert rc == C.OK, C.strerror(rc)
    torch.cuda.synchronize()
    return d_rep.cpu().numpy().view(C.DREPLY_DTYPE).copy()


def test_no_alloc_entry_matches_runtime_entry_on_two_calls():
    wl = W.config1()
    first = np.concatenate([wl.n[:200], np.array(EDGE, dtype=np.uint64)])
    second = np.concatenate([np.array(EDGE[::-1], dtype=np.uint64), wl.n[::-1][:150]])
    with C.Runtime(max_factor_n=MAX40, max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        want = [device_batch(rt, np.full(v.size, a - 1, np.uint32), C.FACTOR_U64, v) for v in (first, second)]
    for values, ref in zip((first, second), want):
        got = _static_call(values)
        assert np.all(got["done"] == 1)
        assert np.array_equal(got["status"], ref["status"])
        assert np.array_equal(got["r0"], ref["r0"])
        assert np.array_equal(got["r1"], ref["r1"])


def test_no_alloc_entry_rejects_oversize_batch():
    # nothing is launched for an oversize batch, so the pointers are never used
    rc = C.factor_static(16, C.FACTOR_STATIC_MAX + 1, 16, 0)
    assert rc == C.EINVAL
