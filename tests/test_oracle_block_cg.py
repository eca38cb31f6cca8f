"""Pins for the oracle's block CG (O'Leary) (CPU only).

Independent checks: with s = 1 it is CG (the oracle's CG, itself pinned); after
k block steps X_k minimises the A-norm error over X_0 + K_k(A, R_0), the block
Krylov space (numpy: explicit basis, Galerkin solve), which no single-column
CG reaches; with n = s m it terminates within m steps (the block Krylov space
fills R^n); the solution is the LAPACK one; dependent columns break down.
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _block_krylov_minimiser(A, B, X0, k):
    R0 = B - A @ X0
    blocks = [R0]
    for _ in range(k - 1):
        blocks.append(A @ blocks[-1])
    V = np.linalg.qr(np.hstack(blocks))[0]
    # Galerkin / A-norm minimiser: V^T A V C = V^T R0
    C = np.linalg.solve(V.T @ A @ V, V.T @ R0)
    return X0 + V @ C


def test_block_cg_s1_is_cg(oracle):
    n = 80
    A = inputs.spd_matrix(n, 0.1, seed=4)
    b = A @ inputs.solution(n, seed=4)
    for k in (1, 3, 9):
        bl = oracle.block_cg(A, b[:, None], rtol=1e-300, max_iter=k)
        cg = oracle.cg(A, b, rtol=1e-300, max_iter=k)
        assert bl["iters"] == cg["iters"] == k
        assert np.allclose(bl["X"][:, 0], cg["x"], rtol=0, atol=1e-12 * np.abs(cg["x"]).max())


@pytest.mark.parametrize("s,k", [(2, 3), (4, 2), (3, 5)])
def test_block_cg_is_block_krylov_minimiser(oracle, s, k):
    n = 40
    A = inputs.spd_matrix(n, 0.5, seed=11)
    B = A @ inputs.solution(n, seed=12, nrhs=s)
    out = oracle.block_cg(A, B, rtol=1e-300, max_iter=k)
    assert out["iters"] == k
    ref = _block_krylov_minimiser(A, B, np.zeros((n, s)), k)
    assert np.max(np.abs(out["X"] - ref)) <= 1e-9 * np.max(np.abs(ref))
    # strictly better than s independent CG runs of k steps (each column alone)
    Xs = np.linalg.solve(A, B)
    e_block = np.trace((out["X"] - Xs).T @ A @ (out["X"] - Xs))
    e_cols = 0.0
    for j in range(s):
        xj = oracle.cg(A, B[:, j], rtol=1e-300, max_iter=k)["x"]
        e_cols += (xj - Xs[:, j]) @ A @ (xj - Xs[:, j])
    assert e_block < e_cols


def test_block_cg_terminates_in_n_over_s_steps(oracle):
    n, s = 24, 6
    A = inputs.spd_matrix(n, 1.0, seed=5)
    B = A @ inputs.solution(n, seed=6, nrhs=s)
    out = oracle.block_cg(A, B, rtol=1e-9, max_iter=100)
    assert out["status"] == oracle.OK and out["iters"] <= n // s


@pytest.mark.parametrize("n,s", [(1, 1), (50, 3), (300, 8)])
def test_block_cg_matches_lapack(oracle, n, s):
    A = inputs.spd_matrix(n, 0.1, seed=30 + n)
    Xs = inputs.solution(n, seed=31 + n, nrhs=s).reshape(n, s)
    B = A @ Xs
    out = oracle.block_cg(A, B, rtol=1e-11)
    assert out["status"] == oracle.OK and out["rel_res"] <= 1e-11
    ref = np.linalg.solve(A, B)
    assert np.max(np.abs(out["X"] - ref)) <= 100 * np.linalg.cond(A) * 1e-11 * np.max(np.abs(ref))


def test_block_cg_breakdown_and_limit(oracle):
    n = 30
    A = inputs.spd_matrix(n, 0.5, seed=8)
    b = A @ inputs.solution(n, seed=8)
    assert oracle.block_cg(A, np.stack([b, b], 1))["status"] == oracle.BREAKDOWN
    assert oracle.block_cg(A, np.stack([b, np.zeros(n)], 1))["status"] == oracle.BREAKDOWN
    B = A @ inputs.solution(n, seed=9, nrhs=3)
    out = oracle.block_cg(A, B, rtol=1e-300, max_iter=2)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 2
