"""Pins for the oracle's Gauss-Seidel iteration (CPU only).

Independent checks: on a lower-triangular matrix one sweep is forward
substitution (scipy's triangular solve); on an upper-triangular one the
iteration matrix is nilpotent, so n sweeps reach the solution; the
fixed point is the LAPACK solution; the asymptotic residual contraction
equals the spectral radius of -(D + L)^-1 U (numpy eigenvalues); Gauss-Seidel
converges on an SPD matrix on which Jacobi diverges (the textbook theorem);
a zero diagonal entry is a breakdown; b = 0 and the iteration limit.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_1511_07207_gb300 import inputs


def _rho_gs(A):
    DL = np.tril(A)
    U = np.triu(A, 1)
    return np.max(np.abs(np.linalg.eigvals(np.linalg.solve(DL, U))))


def test_gs_lower_triangular_is_forward_substitution(oracle):
    n = 30
    A = np.tril(inputs.nonsym_matrix(n, seed=1))
    b = inputs.solution(n, seed=2)
    out = oracle.gauss_seidel(A, b, rtol=1e-15)
    assert out["status"] == oracle.OK and out["iters"] == 2     # one sweep, then the test
    ref = scipy.linalg.solve_triangular(A, b, lower=True)
    assert np.allclose(out["x"], ref, rtol=1e-14, atol=0)


def test_gs_upper_triangular_nilpotent(oracle):
    n = 12
    A = np.triu(inputs.nonsym_matrix(n, seed=3))
    b = inputs.solution(n, seed=4)
    out = oracle.gauss_seidel(A, b, rtol=1e-13, max_iter=2 * n)
    assert out["status"] == oracle.OK and out["iters"] <= n + 1
    ref = scipy.linalg.solve_triangular(A, b, lower=False)
    assert np.allclose(out["x"], ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [1, 3, 40, 200])
def test_gs_matches_lapack(oracle, n):
    A = inputs.nonsym_matrix(n, seed=800 + n)
    b = A @ inputs.solution(n, seed=800 + n)
    out = oracle.gauss_seidel(A, b, rtol=1e-12)
    assert out["status"] == oracle.OK
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(out["x"] - ref) <= 4 * np.linalg.cond(A) * 1e-12 * np.linalg.norm(ref)


def test_gs_rate_is_spectral_radius(oracle):
    n = 120
    A = inputs.restart_matrix(n, seed=5)            # a slower case: rate well inside (0, 1)
    rho = _rho_gs(A)
    assert 0.2 < rho < 0.95
    b = A @ inputs.solution(n, seed=5)
    out = oracle.gauss_seidel(A, b, rtol=1e-14, history=True)
    h = out["res_hist"]
    tail = h[len(h) // 2:]
    rate = (tail[-1] / tail[0]) ** (1.0 / (len(tail) - 1))
    assert abs(rate - rho) <= 0.1 * rho


def test_gs_converges_on_spd_where_jacobi_diverges(oracle):
    n = 60
    A = inputs.spd_matrix(n, 0.5, seed=3)
    d = np.diag(A)
    rho_j = np.max(np.abs(np.linalg.eigvals(np.eye(n) - A / d[:, None])))
    assert rho_j > 1.0 and _rho_gs(A) < 1.0
    b = A @ inputs.solution(n, seed=3)
    assert oracle.gauss_seidel(A, b, rtol=1e-10)["status"] == oracle.OK
    assert oracle.jacobi(A, b, rtol=1e-10, max_iter=300)["status"] != oracle.OK


def test_gs_breakdown_and_limits(oracle):
    A2 = np.eye(3)
    A2[2, 2] = 0.0
    out = oracle.gauss_seidel(A2, np.ones(3), x0=np.full(3, 0.5))
    assert out["status"] == oracle.BREAKDOWN and np.array_equal(out["x"], np.full(3, 0.5))
    A3 = inputs.nonsym_matrix(20, seed=1)
    out = oracle.gauss_seidel(A3, np.zeros(20), x0=np.ones(20))
    assert out["status"] == oracle.OK and not out["x"].any() and out["iters"] == 0
    out = oracle.gauss_seidel(A3, A3 @ inputs.solution(20, seed=1), rtol=1e-300, max_iter=3)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 3
