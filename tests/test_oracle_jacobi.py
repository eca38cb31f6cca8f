"""Pins for the oracle's Jacobi iteration (CPU only).

Independent checks: the fixed point is the LAPACK solution; the asymptotic
contraction of the residual equals the spectral radius of the iteration
matrix I - D^-1 A (numpy eigenvalues), as the power method predicts; a
diagonal matrix is solved by the first update; an iteration matrix of
spectral radius above one does not converge; a zero diagonal entry is a
breakdown; b = 0 and the iteration limit.
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _rho(A):
    d = np.diag(A)
    return np.max(np.abs(np.linalg.eigvals(np.eye(len(d)) - A / d[:, None])))


@pytest.mark.parametrize("n", [1, 3, 40, 200])
def test_jacobi_matches_lapack(oracle, n):
    A = inputs.nonsym_matrix(n, seed=500 + n)
    b = A @ inputs.solution(n, seed=500 + n)
    out = oracle.jacobi(A, b, rtol=1e-12)
    assert out["status"] == oracle.OK
    ref = np.linalg.solve(A, b)
    kap = np.linalg.cond(A)
    assert np.linalg.norm(out["x"] - ref) <= 4 * kap * 1e-12 * np.linalg.norm(ref)
    assert out["rel_res"] <= 1e-12


def test_jacobi_rate_is_spectral_radius(oracle):
    n = 120
    A = inputs.nonsym_matrix(n, seed=7)
    b = A @ inputs.solution(n, seed=7)
    out = oracle.jacobi(A, b, rtol=1e-14, history=True)
    h = out["res_hist"]
    assert len(h) >= 12
    tail = h[len(h) // 2:]
    rate = (tail[-1] / tail[0]) ** (1.0 / (len(tail) - 1))
    assert abs(rate - _rho(A)) <= 0.1 * _rho(A)


def test_jacobi_diagonal_one_update(oracle):
    d = np.array([2.0, -3.0, 0.5, 4.0])
    b = np.array([1.0, 2.0, 3.0, 4.0])
    out = oracle.jacobi(np.diag(d), b, rtol=1e-14)
    assert out["status"] == oracle.OK and out["iters"] == 2      # one update, one test
    assert np.allclose(out["x"], b / d, rtol=0, atol=1e-15)


def test_jacobi_divergence_breakdown_limits(oracle):
    n = 60
    A = inputs.spd_matrix(n, 0.01, seed=3)      # rho(I - D^-1 A) > 1
    assert _rho(A) > 1.0
    b = A @ inputs.solution(n, seed=3)
    out = oracle.jacobi(A, b, rtol=1e-10, max_iter=200)
    assert out["status"] != oracle.OK
    A2 = np.eye(3)
    A2[1, 1] = 0.0
    assert oracle.jacobi(A2, np.ones(3))["status"] == oracle.BREAKDOWN
    A3 = inputs.nonsym_matrix(20, seed=1)
    assert oracle.jacobi(A3, np.zeros(20))["status"] == oracle.OK
    out = oracle.jacobi(A3, A3 @ inputs.solution(20, seed=1), rtol=1e-14, max_iter=3)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 3


def test_jacobi_limit_returns_measured_iterate(oracle):
    # after max_iter products the iterate returned is the last one measured:
    # x(2) = x(1) + D^-1 (b - A x(1)) written out for a 2 x 2 system
    A = np.array([[4.0, 1.0], [2.0, 5.0]])
    b = np.array([1.0, 2.0])
    d = np.diag(A)
    x1 = b / d
    x2 = x1 + (b - A @ x1) / d
    out = oracle.jacobi(A, b, rtol=1e-300, max_iter=3, history=True)
    assert out["iters"] == 3 and out["status"] == oracle.NOT_CONVERGED
    assert np.allclose(out["x"], x2, rtol=0, atol=1e-15)
    assert out["rel_res"] == pytest.approx(np.linalg.norm(b - A @ x2) / np.linalg.norm(b), rel=1e-12)
    assert out["res_hist"][-1] == pytest.approx(np.linalg.norm(b - A @ x2), rel=1e-12)
