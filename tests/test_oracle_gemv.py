"""Direct pins for the oracle's matrix-vector product and residual (CPU only).

Independent checks: on small integers every product and partial sum is exact,
so y = A x and r = b - A x equal numpy's integer arithmetic bit for bit, for
square and rectangular shapes; on random data the product lies within the
classical bound gamma_n |A||x| of the exact one (computed here with Python
fractions); each row is summed left to right, which a row built to cancel
shows; the thread count only splits rows, so the bits do not depend on it.
"""
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -53


def _ints(shape, seed):
    return np.random.default_rng(seed).integers(-8, 9, size=shape).astype(np.float64)


@pytest.mark.parametrize("m,n", [(1, 1), (7, 300), (300, 7), (257, 257)])
def test_gemv_exact_on_integers(oracle, m, n):
    A, x = _ints((m, n), 1 + m), _ints(n, 2 + n)
    y = oracle.gemv(A, x)
    ref = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.float64)
    assert np.array_equal(y, ref)


def test_residual_exact_on_integers(oracle):
    n = 200
    A, x, b = _ints((n, n), 3), _ints(n, 4), _ints(n, 5)
    r = oracle.residual(A, b, x)
    ref = (b.astype(np.int64) - A.astype(np.int64) @ x.astype(np.int64)).astype(np.float64)
    assert np.array_equal(r, ref)
    assert np.array_equal(oracle.residual(A, A @ x, x), np.zeros(n))


def test_gemv_within_the_rounding_bound(oracle):
    m, n = 40, 60
    rng = np.random.default_rng(6)
    A, x = rng.standard_normal((m, n)), rng.standard_normal(n)
    y = oracle.gemv(A, x)
    gamma = n * U / (1 - n * U)
    bound = gamma * (np.abs(A) @ np.abs(x))
    for i in range(m):
        exact = sum((Fraction(a) * Fraction(v) for a, v in zip(A[i], x)), Fraction(0))
        assert abs(Fraction(y[i]) - exact) <= Fraction(bound[i])


def test_rows_summed_left_to_right(oracle):
    # 1 + 2^53 rounds back to 2^53 (ties to even), so left to right the row gives 0, not 1
    A = np.array([[1.0, 2.0 ** 53, -(2.0 ** 53)], [2.0 ** 53, -(2.0 ** 53), 1.0]])
    y = oracle.gemv(A, np.ones(3))
    assert y[0] == 0.0 and y[1] == 1.0


def test_thread_count_does_not_change_the_bits(oracle):
    n = 333
    rng = np.random.default_rng(7)
    A, x, b = rng.standard_normal((n, n)), rng.standard_normal(n), rng.standard_normal(n)
    nt = max(2, oracle.max_threads())
    assert np.array_equal(oracle.gemv(A, x, nthreads=1), oracle.gemv(A, x, nthreads=nt))
    assert np.array_equal(oracle.residual(A, b, x, nthreads=1), oracle.residual(A, b, x, nthreads=nt))
