"""The integer square root shared by the host's prime-table limit and the
device's per-message bounds (csrc/isqrt.h), compiled here for the host with
g++ and checked against Python's exact math.isqrt."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from paper_1505_07368_gb300 import workloads as W

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1505_07368_gb300", "csrc")


@pytest.fixture(scope="module")
def isqrt(tmp_path_factory):
    d = tmp_path_factory.mktemp("isqrt")
    src = d / "t.cpp"
    src.write_text('#include "isqrt.h"\nextern "C" uint64_t t_isqrt(uint64_t n) { return cafgpu::isqrt_u64(n); }\n')
    lib = d / "libt.so"
    subprocess.check_call(["g++", "-O2", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(lib)])
    L = ctypes.CDLL(str(lib))
    L.t_isqrt.argtypes = [ctypes.c_uint64]
    L.t_isqrt.restype = ctypes.c_uint64
    return lambda n: int(L.t_isqrt(n))


def test_edges(isqrt):
    for n in [0, 1, 2, 3, 4, 8, 9, 10, (1 << 62) - 1, 1 << 62, (1 << 64) - 1, (1 << 32) - 1, 1 << 32,
              (1 << 56) - 1, ((1 << 31) - 1) ** 2, ((1 << 32) - 1) ** 2]:
        assert isqrt(n) == math.isqrt(n), n


def test_every_small_n(isqrt):
    for n in range(1 << 14):
        assert isqrt(n) == math.isqrt(n), n


def test_squares_and_neighbours(isqrt):
    ks = [int(k) for k in W.u64(W.stream_key(99, 1), 0, 3000) >> np.uint64(32)]
    ks += [(1 << 31) - 1, 1 << 31, (1 << 31) + 1, 3037000499, (1 << 28) - 57]
    for k in ks:
        for n in (k * k - 1, k * k, k * k + 1, k * k + 2 * k, (k + 1) * (k + 1) - 1):
            if 0 <= n < (1 << 64):
                assert isqrt(n) == math.isqrt(n), n


def test_random_full_range(isqrt):
    for n in W.u64(W.stream_key(99, 2), 0, 5000):
        assert isqrt(int(n)) == math.isqrt(int(n))
