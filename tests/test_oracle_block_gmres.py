"""Pins for the oracle's restarted block GMRES (CPU only).

Independent checks: after k block steps of the first cycle the iterate is the
least-squares minimiser of ||B - A X||_F over X_0 + K_k(A, R_0), the block
Krylov space (numpy: explicit basis, lstsq); with s = 1 it is the oracle's
GMRES (itself pinned); with n = s m' it terminates within m' block steps;
restarted runs reach the LAPACK solution; a rank-deficient right-hand side
block breaks down.
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _block_lsq(A, B, X0, k):
    R0 = B - A @ X0
    blocks = [R0]
    for _ in range(k - 1):
        blocks.append(A @ blocks[-1])
    V = np.linalg.qr(np.hstack(blocks))[0]
    C = np.linalg.lstsq(A @ V, R0, rcond=None)[0]
    return X0 + V @ C


@pytest.mark.parametrize("s,k", [(2, 3), (3, 4), (4, 2)])
def test_block_gmres_is_block_krylov_minimiser(oracle, s, k):
    n = 40
    A = inputs.restart_matrix(n, seed=21)
    B = A @ inputs.solution(n, seed=22, nrhs=s)
    out = oracle.block_gmres(A, B, m=6, rtol=1e-300, max_iter=k)
    assert out["iters"] == k and out["cycles"] == 1
    ref = _block_lsq(A, B, np.zeros((n, s)), k)
    assert np.max(np.abs(out["X"] - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_block_gmres_s1_is_gmres(oracle):
    n = 70
    A = inputs.restart_matrix(n, seed=5)
    b = A @ inputs.solution(n, seed=5)
    for k in (1, 4, 13):
        bl = oracle.block_gmres(A, b[:, None], m=8, rtol=1e-300, max_iter=k)
        gm = oracle.gmres(A, b, m=8, rtol=1e-300, max_iter=k)
        assert bl["iters"] == gm["iters"] == k
        assert np.allclose(bl["X"][:, 0], gm["x"], rtol=0, atol=1e-10 * np.abs(gm["x"]).max())


def test_block_gmres_terminates_in_n_over_s_steps(oracle):
    n, s = 24, 4
    A = inputs.restart_matrix(n, seed=7)
    B = A @ inputs.solution(n, seed=8, nrhs=s)
    out = oracle.block_gmres(A, B, m=n // s, rtol=1e-9)
    assert out["status"] == oracle.OK and out["iters"] <= n // s and out["cycles"] == 1


@pytest.mark.parametrize("n,s,m", [(1, 1, 3), (60, 3, 4), (300, 8, 10)])
def test_block_gmres_matches_lapack(oracle, n, s, m):
    A = inputs.nonsym_matrix(n, seed=40 + n)
    B = A @ inputs.solution(n, seed=41 + n, nrhs=s).reshape(n, s)
    out = oracle.block_gmres(A, B, m=m, rtol=1e-11)
    assert out["status"] == oracle.OK and out["rel_res"] <= 1e-11
    ref = np.linalg.solve(A, B)
    assert np.max(np.abs(out["X"] - ref)) <= 100 * np.linalg.cond(A) * 1e-11 * np.max(np.abs(ref))


def test_block_gmres_breakdown_and_limit(oracle):
    n = 30
    A = inputs.nonsym_matrix(n, seed=9)
    b = A @ inputs.solution(n, seed=9)
    assert oracle.block_gmres(A, np.stack([b, 2 * b], 1), m=5)["status"] == oracle.BREAKDOWN
    B = A @ inputs.solution(n, seed=10, nrhs=3)
    out = oracle.block_gmres(A, B, m=2, rtol=1e-300, max_iter=3)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 3 and out["cycles"] == 2
    out = oracle.block_gmres(A, np.zeros((n, 2)), m=3)
    assert out["status"] == oracle.OK and out["iters"] == 0 and not out["X"].any()
