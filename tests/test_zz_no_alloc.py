"""caf_gpu_factor_static: the factorization call that allocates no device memory.

It is meant for callers that cannot call cudaMalloc (a host framework whose
allocator owns the GPU's memory, latency-critical paths, programs that forbid
allocation after start-up).  This test calls it through the C ABI, twice in a
row with different numbers (so a stale scratch word from the first call would
show in the second), and requires the same replies as the runtime's device
batch entry point and as the CPU oracle's trial division.  The file is named
to be collected last.
"""
import numpy as np
import pytest

from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

import oracle
from helpers import device_batch

pytestmark = pytest.mark.gpu

MAX40 = (1 << 40) - 1
EDGE = [0, 1, 2, 3, 4, 5, 8, 9, 15, 25, 49, 97 * 97, 1 << 39, MAX40, 1048573 * 1048573,
        1048573 * 1048571, 1048573, 999983 * 2, 3 * 1048573, (1 << 40) - 87]


def _largest_primes_below(x: int, k: int):
    out, c = [], x - 1 if x % 2 == 0 else x - 2
    while len(out) < k:
        if oracle.is_prime(c):
            out.append(c)
        c -= 2
    return out


# odd primes just below 2^40 (every candidate up to the root is tried) and
# squares of the primes just below 2^20 (the divisor is the root itself)
PRIMES40 = _largest_primes_below(1 << 40, 4)
SQUARES40 = [p * p for p in _largest_primes_below(1 << 20, 4)]


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
    extra = np.array(EDGE + PRIMES40 + SQUARES40, dtype=np.uint64)
    first = np.concatenate([wl.n[:200], extra])
    second = np.concatenate([extra[::-1], wl.n[::-1][:150]])
    with C.Runtime(max_factor_n=MAX40, max_actors=4) as rt:
        a = rt.spawn(C.FACTOR_U64)
        want = [device_batch(rt, np.full(v.size, a - 1, np.uint32), C.FACTOR_U64, v) for v in (first, second)]
    for values, ref in zip((first, second), want):
        got = _static_call(values)
        assert np.all(got["done"] == 1)
        assert np.array_equal(got["status"], ref["status"])
        assert np.array_equal(got["r0"], ref["r0"])
        assert np.array_equal(got["r1"], ref["r1"])
        st, p, q = oracle.factor_batch(values)
        assert np.array_equal(got["status"], st)
        assert np.array_equal(got["r0"], p) and np.array_equal(got["r1"], q)


def test_no_alloc_entry_beyond_the_runtime_default_range():
    # n up to 2^50 and values at and past the 2^62 limit, against the oracle
    big = _largest_primes_below(1 << 50, 2) + [((1 << 25) - 39) * ((1 << 25) - 39), (1 << 62) - 2,
                                                 3 * ((1 << 60) + 1)]
    values = np.array(big, dtype=np.uint64)
    got = _static_call(values)
    st, p, q = oracle.factor_batch(values)
    assert np.array_equal(got["status"], st)
    assert np.array_equal(got["r0"], p) and np.array_equal(got["r1"], q)
    rej = _static_call(np.array([1 << 62, (1 << 64) - 1], dtype=np.uint64))
    assert np.all(rej["status"] == C.REPLY_REJECTED)


def test_no_alloc_entry_rejects_oversize_batch():
    # nothing is launched for an oversize batch, so the pointers are never used
    rc = C.factor_static(16, C.FACTOR_STATIC_MAX + 1, 16, 0)
    assert rc == C.EINVAL
