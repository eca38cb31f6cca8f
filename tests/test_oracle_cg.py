"""Pins for the oracle's conjugate gradient (CPU only).

Each check uses mathematics that does not depend on the oracle's code:
LAPACK solves, the Krylov optimality of CG (the k-th iterate minimises the
A-norm of the error over K_k(A, b), computed here by a Galerkin projection
on an explicit basis), finite termination for k distinct eigenvalues,
mutual orthogonality of residuals and A-conjugacy of directions, and the
classical sqrt(kappa) iteration bound.
"""
import math

import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _krylov_galerkin(A, b, k):
    """A-norm-optimal x in K_k(A, b): orthonormal basis by QR, then Galerkin."""
    K = np.empty((A.shape[0], k))
    v = b / np.linalg.norm(b)
    for j in range(k):
        K[:, j] = v
        v = A @ v
        v = v / np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    y = np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
    return Q @ y


@pytest.mark.parametrize("n", [64, 200, 512])
def test_cg_matches_lapack(oracle, n):
    A = inputs.spd_matrix(n, 0.1, seed=n)
    xs = inputs.solution(n, seed=n)
    b = A @ xs
    out = oracle.cg(A, b, rtol=1e-10)
    assert out["status"] == oracle.OK
    x_ref = np.linalg.solve(A, b)
    rel_res = np.linalg.norm(b - A @ out["x"]) / np.linalg.norm(b)
    assert rel_res <= 1e-10
    assert abs(rel_res - out["rel_res"]) <= 1e-3 * rel_res + 1e-18
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    err = np.linalg.norm(out["x"] - x_ref) / np.linalg.norm(x_ref)
    assert err <= 2 * kappa * 1e-10
    # classical bound: iters <= ceil(sqrt(kappa)/2 * ln(2/tol))
    assert out["iters"] <= math.ceil(0.5 * math.sqrt(kappa) * math.log(2 / 1e-10))


def test_cg_krylov_optimality(oracle):
    n = 48
    A = inputs.spd_matrix(n, 0.05, seed=7)
    b = A @ inputs.solution(n, seed=7)
    for k in range(1, 9):
        out = oracle.cg(A, b, rtol=0.0, max_iter=k)
        assert out["iters"] == k
        x_opt = _krylov_galerkin(A, b, k)
        assert np.linalg.norm(out["x"] - x_opt) <= 1e-9 * np.linalg.norm(x_opt)


@pytest.mark.parametrize("eigs", [[1.0, 2.0, 3.0, 4.0, 5.0], [0.5, 7.0, 30.0]])
def test_cg_distinct_eigenvalues_terminate(oracle, eigs):
    n = 60
    A = inputs.distinct_eig_spd(n, eigs, seed=3)
    b = A @ inputs.solution(n, seed=3)
    out = oracle.cg(A, b, rtol=1e-10)
    assert out["status"] == oracle.OK
    assert out["iters"] == len(eigs)


def test_cg_orthogonality_and_conjugacy(oracle):
    n = 30
    A = inputs.spd_matrix(n, 0.5, seed=11)
    b = A @ inputs.solution(n, seed=11)
    out = oracle.cg(A, b, rtol=1e-14, max_iter=8, history=True)
    R, P = out["R"][:8], out["P"][:8]
    for i in range(8):
        for j in range(i):
            c = abs(R[i] @ R[j]) / (np.linalg.norm(R[i]) * np.linalg.norm(R[j]))
            assert c <= 1e-8, (i, j, c)
            d = abs(P[i] @ A @ P[j]) / math.sqrt((P[i] @ A @ P[i]) * (P[j] @ A @ P[j]))
            assert d <= 1e-8, (i, j, d)
    # residual norms recorded match the true ones of the recurrence
    assert np.allclose(out["res_hist"][:8], np.linalg.norm(R, axis=1), rtol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 32])
def test_cg_finite_termination_small(oracle, n):
    A = inputs.spd_matrix(n, 1.0, seed=100 + n)  # cond <= ~5
    b = A @ inputs.solution(n, seed=100 + n)
    out = oracle.cg(A, b, rtol=1e-12, max_iter=n)
    assert out["status"] == oracle.OK
    assert out["iters"] <= n
    assert np.linalg.norm(b - A @ out["x"]) <= 1e-12 * np.linalg.norm(b)


def test_cg_edge_cases(oracle):
    n = 10
    A = inputs.spd_matrix(n, 1.0, seed=1)
    out = oracle.cg(A, np.zeros(n))
    assert out["status"] == oracle.OK and out["iters"] == 0 and not out["x"].any()
    # an exact start needs no iteration
    xs = inputs.solution(n, seed=1)
    out = oracle.cg(np.eye(n) * 3.0, 3.0 * xs, x0=xs)
    assert out["status"] == oracle.OK and out["iters"] == 0
    # negative definite: curvature p.Ap <= 0 is a breakdown, not a crash
    out = oracle.cg(-A, A @ xs)
    assert out["status"] == oracle.BREAKDOWN
    # max_iter reached without convergence
    B = inputs.spd_matrix(200, 1e-3, seed=2)
    out = oracle.cg(B, B @ inputs.solution(200, seed=2), rtol=1e-12, max_iter=3)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 3


def test_cg_threads_do_not_change_results(oracle):
    n = 300
    A = inputs.spd_matrix(n, 0.1, seed=5)
    b = A @ inputs.solution(n, seed=5)
    a = oracle.cg(A, b, nthreads=1)
    c = oracle.cg(A, b, nthreads=4)
    assert a["iters"] == c["iters"]
    assert np.array_equal(a["x"], c["x"])
