"""Validation mode's memory checks, exercised by host-side injection only (no
device fault is made): the guard regions after every device array stay
intact through real workloads, a mailbox pointed past the slot pool is refused
by the device's bounds check before anything is read or written there, and an
overwritten guard is reported."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import device_batch

pytestmark = pytest.mark.gpu


def test_guards_intact_after_factor_ring_and_gemm_work():
    import torch
    wl = W.config1()
    with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=16, validation_mode=1) as rt:
        f = rt.spawn(C.FACTOR_U64)
        rep = device_batch(rt, np.full(wl.count, f - 1, np.uint32), C.FACTOR_U64, wl.n)
        st, p, q = oracle.factor_batch(wl.n)
        assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q)
        g = rt.spawn(C.GEMM_SPLIT_BF16X3)
        n = 200
        A = torch.randn(n, n, device="cuda")
        B = torch.randn(n, n, device="cuda")
        Cm = torch.empty(n, n, device="cuda")
        h = rt.request(g, C.Runtime.msg(C.GEMM_SPLIT_BF16X3, n=n, A=A.data_ptr(), B=B.data_ptr(), C=Cm.data_ptr()))
        assert rt.await_(h, 60_000_000_000)[0] == 0
        assert rt.check_guards() == 0


def test_injected_out_of_range_mailbox_is_refused():
    wl = W.config1()
    with C.Runtime(max_factor_n=(1 << 40) - 1, max_actors=4, validation_mode=1) as rt:
        bad = rt.spawn(C.FACTOR_U64)
        good = rt.spawn(C.FACTOR_U64)
        assert rt.debug_inject(1, bad) == C.OK
        with pytest.raises(C.CafGpuError) as e:
            device_batch(rt, np.full(4, bad - 1, np.uint32), C.FACTOR_U64, wl.n[:4])
        assert e.value.code == C.EBOUNDS
        st = rt.stats()
        assert st["error_word"] & 0xFF == 10 and (st["error_word"] >> 8) == 40   # refused at the enqueue
        assert st["diag0"] == bad - 1
        rt.clear_error()
        # the runtime goes on serving the other actor, and nothing was overwritten
        rep = device_batch(rt, np.full(8, good - 1, np.uint32), C.FACTOR_U64, wl.n[:8])
        _, p, q = oracle.factor_batch(wl.n[:8])
        assert np.array_equal(rep["r0"], p) and np.array_equal(rep["r1"], q)
        assert rt.check_guards() == 0


def test_injection_needs_validation_mode_and_overwritten_guard_is_reported():
    rt = C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=4)
    try:
        a = rt.spawn(C.FACTOR_U64)
        assert rt.debug_inject(1, a) == C.EINVAL        # no bounds checks without validation mode
        assert rt.debug_inject(3, 0) == C.EINVAL
        assert rt.check_guards() == 0
        assert rt.debug_inject(2, 0) == C.OK
        assert rt.check_guards() == 1
    finally:
        with pytest.raises(C.CafGpuError) as e:
            rt.close()
    assert e.value.code == C.EBOUNDS
