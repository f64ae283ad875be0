"""Pins for the oracle's float64 matrix product and the Frobenius error."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 96])
def test_integer_matrices_exact(n):
    A = W.integer_matrix(W.stream_key(5, n), n)
    B = W.integer_matrix(W.stream_key(6, n), n)
    want = A.astype(np.int64) @ B.astype(np.int64)
    C = oracle.gemm_f64(A, B)
    assert np.array_equal(C, want.astype(np.float64))


def test_hand_computed_2x2_and_3x3():
    A = np.array([[1, 2], [3, 4]], np.float32)
    B = np.array([[5, 6], [7, 8]], np.float32)
    assert np.array_equal(oracle.gemm_f64(A, B), [[19, 22], [43, 50]])
    A = np.array([[1, 0, 2], [0, 3, 0], [4, 0, 5]], np.float32)
    B = np.array([[0, 1, 0], [2, 0, 0], [0, 0, 3]], np.float32)
    assert np.array_equal(oracle.gemm_f64(A, B), [[0, 1, 6], [6, 0, 0], [0, 4, 15]])


def test_identity_and_permutation():
    n = 33
    A = W.normal_f32(W.stream_key(7, 1), 0, n * n).reshape(n, n)
    I = np.eye(n, dtype=np.float32)
    assert np.array_equal(oracle.gemm_f64(A, I), A.astype(np.float64))
    assert np.array_equal(oracle.gemm_f64(I, A), A.astype(np.float64))
    P = np.eye(n, dtype=np.float32)[::-1].copy()
    assert np.array_equal(oracle.gemm_f64(P, A), A[::-1].astype(np.float64))


def test_random_against_numpy_blas():
    n = 80
    A = W.normal_f32(W.stream_key(8, 1), 0, n * n).reshape(n, n)
    B = W.normal_f32(W.stream_key(8, 2), 0, n * n).reshape(n, n)
    C = oracle.gemm_f64(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64)
    assert np.max(np.abs(C - ref)) <= 1e-12 * np.max(np.abs(ref))
    for (i, j) in [(0, 0), (5, 79), (79, 3)]:
        assert oracle.gemm_entry(A, B, i, j) == C[i, j]


def test_rel_frobenius_closed_forms():
    C64 = np.array([3.0, 4.0])
    assert oracle.rel_frobenius(np.array([3, 4], np.float32), C64) == 0.0
    assert oracle.rel_frobenius(np.array([0, 0], np.float32), C64) == 1.0
    assert oracle.rel_frobenius(np.array([6, 8], np.float32), C64) == 1.0
    assert abs(oracle.rel_frobenius(np.array([3, 4.5], np.float32), C64) - 0.1) < 1e-15
    assert oracle.rel_frobenius(np.array([0, 0], np.float32), np.zeros(2)) == 0.0


@pytest.mark.parametrize("n", [5, 64, 129, 1100])
def test_rows_integer_matrices_exact(n):
    # integer entries in [-8, 8]: every partial sum is an integer below 2^53,
    # so the selected rows must equal the int64 product's rows exactly
    A = W.integer_matrix(W.stream_key(9, n), n)
    B = W.integer_matrix(W.stream_key(10, n), n)
    rows = np.unique(np.array([0, n - 1, n // 2, min(n - 1, 127), min(n - 1, 128)], np.int64))
    want = A[rows].astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(oracle.gemm_rows(A, B, rows), want.astype(np.float64))


def test_rows_pick_rows_and_not_columns():
    # a row permutation of A permutes the product's rows: a transposed operand
    # or a row/column mix-up in the row selection fails this
    n = 40
    A = W.normal_f32(W.stream_key(11, 1), 0, n * n).reshape(n, n)
    B = W.normal_f32(W.stream_key(11, 2), 0, n * n).reshape(n, n)
    P = np.eye(n, dtype=np.float32)[np.roll(np.arange(n), 7)].copy()
    rows = np.array([3, 0, 39, 17], np.int64)
    got = oracle.gemm_rows(P @ A, B, rows)
    full = oracle.gemm_f64(A, B)
    assert np.array_equal(got, full[(rows - 7) % n])   # row i of P is e_{i-7}
    assert np.array_equal(oracle.gemm_rows(A, B, rows), full[rows])
    assert oracle.gemm_rows(A, B, np.array([], np.int64)).shape == (0, n)
