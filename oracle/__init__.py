"""CPU oracle for the GPU compute-actor path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package.  It shares no code with the CUDA library: the
numeric payloads live in ``oracle.c`` (plain single-threaded C, loaded
through ctypes) and the actor semantics in ``actors.py`` (plain Python).

Functions and the passages they follow:

* ``factor`` / ``factor_batch`` -- trial division as the plain definition
  of the factorization side load of the mixed benchmark (Sec. 5, "Mixed
  Operations Under Work Load"): smallest d >= 2 with d*d <= n and d | n.
* ``check_certificate`` / ``is_prime`` -- p*q == n, p <= q, p and q prime.
* ``gemm_f64`` / ``gemm_rows`` / ``gemm_entry`` -- the matrix product of the OpenCL actor
  example (Sec. 3.6) in float64 from float32 inputs.
* ``rel_frobenius`` -- relative Frobenius error in float64.
* ``mandel_point`` / ``mandel_rows`` -- escape counts of the Mandelbrot
  iteration in float32 for the OpenCL actor experiment (Sec. 5,
  "Integrating OpenCL Actors").
* ``actors.simulate_mailboxes`` / ``actors.check_mailbox_log`` -- the
  mailbox of Sec. 3.2 and Sec. 2 (FIFO, one reader, exactly-once handling).
* ``actors.simulate_rings`` -- the token rings of Sec. 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, -O2, no -march flags).

    ``-ffp-contract=off``: every float operation is rounded on its own (no
    fused multiply-add), on x86 and on Arm alike."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", _LIB,
                               _SRC, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.oracle_factor.argtypes = [ctypes.c_uint64, u64p, u64p]
        L.oracle_factor.restype = ctypes.c_int32
        L.oracle_factor_batch.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_factor_batch.restype = None
        L.oracle_is_prime.argtypes = [ctypes.c_uint64]
        L.oracle_is_prime.restype = ctypes.c_int32
        L.oracle_check_certificate.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.c_int32]
        L.oracle_check_certificate.restype = ctypes.c_int32
        L.oracle_gemm_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.oracle_gemm_f64.restype = None
        L.oracle_gemm_rows.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p]
        L.oracle_gemm_rows.restype = None
        L.oracle_gemm_entry.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64]
        L.oracle_gemm_entry.restype = ctypes.c_double
        L.oracle_rel_frobenius.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        L.oracle_rel_frobenius.restype = ctypes.c_double
        L.oracle_mandel_point.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_uint32]
        L.oracle_mandel_point.restype = ctypes.c_uint32
        L.oracle_mandel_rows.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_void_p]
        L.oracle_mandel_rows.restype = ctypes.c_uint64
        _lib = L
    return _lib


def factor(n: int):
    """(status, p, q) for one n: status 0 -> n = p*q with p the smallest divisor >= 2
    and p*p <= n; status 1 -> no such divisor, (p, q) = (1, n)."""
    p = ctypes.c_uint64()
    q = ctypes.c_uint64()
    s = lib().oracle_factor(ctypes.c_uint64(int(n)), ctypes.byref(p), ctypes.byref(q))
    return int(s), int(p.value), int(q.value)


def factor_batch(n: np.ndarray):
    """Vector form of ``factor``: returns (status int32, p uint64, q uint64)."""
    n = np.ascontiguousarray(n, dtype=np.uint64)
    p = np.empty_like(n)
    q = np.empty_like(n)
    st = np.empty(n.size, dtype=np.int32)
    lib().oracle_factor_batch(n.ctypes.data, n.size, p.ctypes.data, q.ctypes.data, st.ctypes.data)
    return st, p, q


def is_prime(x: int) -> bool:
    return bool(lib().oracle_is_prime(ctypes.c_uint64(int(x))))


def check_certificate(n: int, p: int, q: int, status: int) -> bool:
    return bool(lib().oracle_check_certificate(int(n), int(p), int(q), int(status)))


def gemm_f64(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n)
    C = np.empty((n, n), dtype=np.float64)
    lib().oracle_gemm_f64(A.ctypes.data, B.ctypes.data, n, C.ctypes.data)
    return C


def gemm_rows(A: np.ndarray, B: np.ndarray, rows) -> np.ndarray:
    """Rows ``rows`` of ``gemm_f64(A, B)`` (float64, shape (len(rows), n)), each
    computed as ``gemm_f64`` computes it; for products too large to form whole."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    n = A.shape[0]
    assert A.shape == (n, n) and B.shape == (n, n)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    assert r.ndim == 1 and (r.size == 0 or (r.min() >= 0 and r.max() < n))
    out = np.empty((r.size, n), dtype=np.float64)
    lib().oracle_gemm_rows(A.ctypes.data, B.ctypes.data, n, r.ctypes.data, r.size, out.ctypes.data)
    return out


def gemm_entry(A: np.ndarray, B: np.ndarray, i: int, j: int) -> float:
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    return float(lib().oracle_gemm_entry(A.ctypes.data, B.ctypes.data, A.shape[0], i, j))


def rel_frobenius(C: np.ndarray, C64: np.ndarray) -> float:
    C = np.ascontiguousarray(C, dtype=np.float32)
    C64 = np.ascontiguousarray(C64, dtype=np.float64)
    assert C.size == C64.size
    return float(lib().oracle_rel_frobenius(C.ctypes.data, C64.ctypes.data, C.size))


def mandel_point(cx: float, cy: float, max_iter: int) -> int:
    """Escape count of c = cx + i cy (both rounded to float32 first)."""
    return int(lib().oracle_mandel_point(float(np.float32(cx)), float(np.float32(cy)), int(max_iter)))


def mandel_rows(x0: float, y0: float, dx: float, dy: float, width: int, row0: int, rows: int, max_iter: int):
    """Escape counts of rows row0 .. row0+rows-1 (pixel (i, j): c = x0 + i dx + (y0 + j dy) i, float32).

    Returns (counts uint32 of shape (rows, width), sum of the counts)."""
    out = np.empty((rows, width), dtype=np.uint32)
    f = [float(np.float32(v)) for v in (x0, y0, dx, dy)]
    s = lib().oracle_mandel_rows(f[0], f[1], f[2], f[3], int(width), int(row0), int(rows), int(max_iter),
                                 out.ctypes.data)
    return out, int(s)
