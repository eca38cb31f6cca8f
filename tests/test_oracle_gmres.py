"""Pins for the oracle's restarted GMRES(m) (CPU only).

Independent checks: the minimal-residual property (the k-th iterate of a
cycle minimises ||b - A x|| over x0 + K_k, computed with numpy lstsq on an
explicit orthonormal Krylov basis), the Arnoldi relation
A V_k = V_{k+1} Hbar_k and orthonormality of V, agreement of the Givens
residual estimate with the true residual, termination within n steps when
m >= n, restart behaviour, and LAPACK solves.
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _krylov_min_residual(A, b, k):
    K = np.empty((A.shape[0], k))
    v = b / np.linalg.norm(b)
    for j in range(k):
        K[:, j] = v
        v = A @ v
        v = v / np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    return Q @ y


def test_gmres_minimal_residual(oracle):
    n = 40
    A = inputs.restart_matrix(n, seed=21)
    b = A @ inputs.solution(n, seed=21)
    for k in range(1, 10):
        out = oracle.gmres(A, b, m=30, rtol=0.0, max_iter=k)
        assert out["iters"] == k and out["cycles"] == 1
        x_opt = _krylov_min_residual(A, b, k)
        r_or = np.linalg.norm(b - A @ out["x"])
        r_opt = np.linalg.norm(b - A @ x_opt)
        assert abs(r_or - r_opt) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(out["x"] - x_opt) <= 1e-8 * np.linalg.norm(x_opt)
        # Givens estimate equals the true residual of the cycle iterate
        assert abs(out["est"] - r_or / np.linalg.norm(b)) <= 1e-12


def test_gmres_residual_monotone_within_cycle(oracle):
    n = 60
    A = inputs.restart_matrix(n, seed=4)
    b = A @ inputs.solution(n, seed=4)
    prev = np.inf
    for k in range(1, 25):
        out = oracle.gmres(A, b, m=30, rtol=0.0, max_iter=k)
        assert out["rel_res"] <= prev * (1 + 1e-12)
        prev = out["rel_res"]


@pytest.mark.parametrize("m", [5, 12])
def test_arnoldi_relation_and_orthonormality(oracle, m):
    n = 80
    A = inputs.nonsym_matrix(n, seed=9)
    b = A @ inputs.solution(n, seed=9)
    out = oracle.gmres(A, b, m=m, rtol=1e-14, first_cycle=True)
    k = out["k"]
    assert k == m
    V, H = out["V"][:, : k + 1], out["H"][: k + 1, :k]
    assert np.linalg.norm(A @ V[:, :k] - V @ H) <= 1e-12 * np.linalg.norm(A)
    assert np.max(np.abs(V.T @ V - np.eye(k + 1))) <= 1e-12
    # Hessenberg structure: zero below the first subdiagonal, positive subdiagonal
    assert np.all(np.tril(H, -2) == 0)
    assert np.all(np.diag(H, -1) > 0)
    # v_1 = r0 / ||r0|| (x0 = 0)
    assert np.allclose(V[:, 0], b / np.linalg.norm(b), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [3, 12, 20])
def test_gmres_terminates_within_n_steps(oracle, n):
    A = inputs.restart_matrix(n, seed=30 + n)
    b = A @ inputs.solution(n, seed=30 + n)
    out = oracle.gmres(A, b, m=n, rtol=1e-12)
    assert out["status"] == oracle.OK
    assert out["iters"] <= n
    assert np.linalg.norm(b - A @ out["x"]) <= 1e-12 * np.linalg.norm(b)


def test_gmres_restarts(oracle):
    n = 200
    A = inputs.restart_matrix(n, seed=13)
    b = A @ inputs.solution(n, seed=13)
    out = oracle.gmres(A, b, m=5, rtol=1e-10, max_iter=5000)
    assert out["status"] == oracle.OK and out["cycles"] > 3
    assert np.linalg.norm(b - A @ out["x"]) <= 1e-10 * np.linalg.norm(b)
    # first cycle = minimal residual over K_5
    one = oracle.gmres(A, b, m=5, rtol=0.0, max_iter=5)
    x_opt = _krylov_min_residual(A, b, 5)
    assert np.linalg.norm(one["x"] - x_opt) <= 1e-9 * np.linalg.norm(x_opt)
    # the true residual never grows from one cycle to the next
    prev = np.inf
    for c in range(1, 8):
        r = oracle.gmres(A, b, m=5, rtol=0.0, max_iter=5 * c)["rel_res"]
        assert r <= prev * (1 + 1e-12)
        prev = r


@pytest.mark.parametrize("n", [64, 512])
def test_gmres_matches_lapack(oracle, n):
    A = inputs.nonsym_matrix(n, seed=n)
    xs = inputs.solution(n, seed=n)
    b = A @ xs
    out = oracle.gmres(A, b, m=30, rtol=1e-10)
    assert out["status"] == oracle.OK
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(b - A @ out["x"]) <= 1e-10 * np.linalg.norm(b)
    s = np.linalg.svd(A, compute_uv=False)
    kappa = s[0] / s[-1]
    assert np.linalg.norm(out["x"] - x_ref) <= 2 * kappa * 1e-10 * np.linalg.norm(x_ref)
    assert out["iters"] < 30   # spectrum in a disk of radius ~1/2 around 2


def test_gmres_lucky_breakdown_and_edges(oracle):
    n = 16
    xs = inputs.solution(n, seed=2)
    out = oracle.gmres(np.eye(n) * 2.0, 2.0 * xs, m=10)
    assert out["status"] == oracle.OK and out["iters"] == 1
    assert np.allclose(out["x"], xs, rtol=0, atol=1e-15)
    D = np.diag(np.arange(1.0, n + 1))
    e = np.zeros(n)
    e[3] = 1.0
    out = oracle.gmres(D, e, m=10)          # b is an eigenvector
    assert out["status"] == oracle.OK and out["iters"] == 1
    out = oracle.gmres(D, np.zeros(n), m=10)
    assert out["status"] == oracle.OK and out["iters"] == 0 and not out["x"].any()
    # singular A with b outside its range: GMRES stagnates, not a false OK
    S = np.diag(np.r_[np.zeros(1), np.ones(n - 1)])
    out = oracle.gmres(S, np.ones(n), m=4, rtol=1e-10, max_iter=40)
    assert out["status"] != oracle.OK
