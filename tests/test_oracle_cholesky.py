"""Pins of the oracle's Cholesky factorization (the paper's direct method
for SPD matrices: A = L L^T, then L y = b and L^T x = y).

Against what does not depend on the oracle: the worked example of
tests/golden/cholesky_3x3.txt (exact), LAPACK's factor (numpy) within
rounding, the backward-error bound |A - L L^T| <= (n + 1) u |L| |L^T|
(Higham, Theorem 10.3), LAPACK solves, uniqueness (L with a positive
diagonal), and the breakdown on matrices that are not positive definite.
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs
from test_oracle_golden import load

U = 2.0 ** -53


def test_cholesky_worked_example(oracle):
    g = load("cholesky_3x3.txt")
    L, st = oracle.chol_factor(g["A"])
    assert st == 0 and np.array_equal(L, g["L"])
    x, st = oracle.chol_solve(g["A"], g["b"])
    assert st == 0 and np.array_equal(x, g["x"])
    assert np.array_equal(oracle.chol_forward(g["L"], g["b"]), g["y"])
    L, st = oracle.chol_factor(g["indefinite_A"])
    assert st == 2


@pytest.mark.parametrize("n", [1, 2, 17, 64, 200])
def test_cholesky_matches_lapack_and_backward_error(oracle, n):
    A = inputs.spd_matrix(n, 0.1, seed=400 + n)
    L, st = oracle.chol_factor(A)
    assert st == 0
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) > 0)
    ref = np.linalg.cholesky(A)
    assert np.max(np.abs(L - ref)) <= 1e-12 * np.max(np.abs(ref))
    bound = (n + 1) * U / (1 - (n + 1) * U) * (np.abs(L) @ np.abs(L.T))
    assert np.all(np.abs(A - L @ L.T) <= bound + 1e-300)


@pytest.mark.parametrize("n", [1, 33, 150])
def test_cholesky_solve_matches_lapack(oracle, n):
    A = inputs.spd_matrix(n, 0.1, seed=500 + n)
    xs = inputs.solution(n, seed=500 + n)
    b = A @ xs
    x, st = oracle.chol_solve(A, b)
    assert st == 0
    ref = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(x - ref) <= 50 * n * kappa * U * np.linalg.norm(ref)


def test_cholesky_reads_only_the_lower_triangle(oracle):
    n = 40
    A = inputs.spd_matrix(n, 0.1, seed=7)
    junk = A.copy()
    junk[np.triu_indices(n, 1)] = 1e30                  # the upper triangle is never read
    L1, s1 = oracle.chol_factor(A)
    L2, s2 = oracle.chol_factor(junk)
    assert s1 == s2 == 0 and np.array_equal(L1, L2)


def test_cholesky_not_positive_definite(oracle):
    rng = np.random.default_rng(3)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.r_[np.ones(n - 1), -1.0]) @ Q.T   # one negative eigenvalue
    A = (A + A.T) / 2
    L, st = oracle.chol_factor(A)
    assert st == 2
    assert oracle.chol_solve(A, np.ones(n))[1] == 2


@pytest.mark.parametrize("n", [1, 5, 80])
def test_cholesky_forward_substitution(oracle, n):
    A = inputs.spd_matrix(n, 0.1, seed=600 + n)
    L, st = oracle.chol_factor(A)
    b = inputs.solution(n, seed=601 + n)
    y = oracle.chol_forward(L, b)
    import scipy.linalg
    ref = scipy.linalg.solve_triangular(L, b, lower=True)
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(L @ y - b)) <= 4 * n * U * np.max(np.abs(L) @ np.abs(y))
