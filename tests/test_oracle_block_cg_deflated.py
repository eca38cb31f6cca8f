"""Pins for the oracle's deflating block CG (CPU only): directions kept
orthonormal and of full rank by a rank-revealing orthogonalization, dependent
ones dropped.

Independent checks: with s = 1 it is CG (the oracle's CG, itself pinned);
with a full-rank block, after k steps X_k is the A-norm minimiser over
X_0 + K_k(A, R_0) (numpy: explicit basis, Galerkin solve), the same iterate
as O'Leary's block CG (pinned the same way); it terminates within n / s
steps when n = s m; solutions are LAPACK's.  What O'Leary's form cannot do:
a block with a zero column, two equal columns, or a column that is a
combination of others converges instead of breaking down; the dependent
column's solution is the same combination of the others' (linearity), the
zero column's is zero; the final rank reports the dropped directions.
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
    C = np.linalg.solve(V.T @ A @ V, V.T @ R0)
    return X0 + V @ C


def test_s1_is_cg(oracle):
    n = 80
    A = inputs.spd_matrix(n, 0.1, seed=4)
    b = A @ inputs.solution(n, seed=4)
    for k in (1, 3, 9, 20):
        bl = oracle.block_cg_deflated(A, b[:, None], rtol=1e-300, max_iter=k)
        cg = oracle.cg(A, b, rtol=1e-300, max_iter=k)
        assert bl["iters"] == cg["iters"] == k and bl["rank"] == 1
        assert np.max(np.abs(bl["X"][:, 0] - cg["x"])) <= 1e-12 * np.abs(cg["x"]).max()


@pytest.mark.parametrize("s,k", [(2, 3), (4, 2), (3, 5)])
def test_full_rank_is_the_block_krylov_minimiser_and_oleary(oracle, s, k):
    n = 40
    A = inputs.spd_matrix(n, 0.5, seed=11)
    B = A @ inputs.solution(n, seed=12, nrhs=s)
    out = oracle.block_cg_deflated(A, B, rtol=1e-300, max_iter=k)
    assert out["iters"] == k and out["rank"] == s
    ref = _block_krylov_minimiser(A, B, np.zeros((n, s)), k)
    assert np.max(np.abs(out["X"] - ref)) <= 1e-9 * np.max(np.abs(ref))
    ol = oracle.block_cg(A, B, rtol=1e-300, max_iter=k)
    assert np.max(np.abs(out["X"] - ol["X"])) <= 1e-9 * np.max(np.abs(ref))


def test_terminates_in_n_over_s_steps(oracle):
    n, s = 24, 6
    A = inputs.spd_matrix(n, 1.0, seed=5)
    B = A @ inputs.solution(n, seed=6, nrhs=s)
    out = oracle.block_cg_deflated(A, B, rtol=1e-9, max_iter=100)
    assert out["status"] == 0 and out["iters"] <= n // s + 1


@pytest.mark.parametrize("n,s", [(60, 3), (200, 8)])
def test_lapack_solutions(oracle, n, s):
    A = inputs.spd_matrix(n, 0.05, seed=30 + n)
    B = A @ inputs.solution(n, seed=31 + n, nrhs=s)
    out = oracle.block_cg_deflated(A, B, rtol=1e-11)
    assert out["status"] == 0 and out["rel_res"] <= 1e-11
    Xl = np.linalg.solve(A, B)
    kap = np.linalg.cond(A)
    assert np.max(np.abs(out["X"] - Xl)) <= 10 * kap * 1e-11 * np.max(np.abs(Xl))


def test_rank_deficient_blocks_converge(oracle):
    n = 120
    A = inputs.spd_matrix(n, 0.1, seed=40)
    X1 = inputs.solution(n, seed=41, nrhs=3)
    B = A @ X1
    # columns: b0, b1, b0 + 2 b1 (dependent), 0, b2, b1 (a duplicate)
    Bd = np.column_stack([B[:, 0], B[:, 1], B[:, 0] + 2 * B[:, 1], np.zeros(n), B[:, 2], B[:, 1]])
    ol = oracle.block_cg(A, Bd, rtol=1e-10)
    assert ol["status"] == 2                              # O'Leary's form breaks down
    out = oracle.block_cg_deflated(A, Bd, rtol=1e-10)
    assert out["status"] == 0 and out["rel_res"] <= 1e-10
    X = out["X"]
    assert not X[:, 3].any()                               # b = 0 -> x = 0
    sc = np.max(np.abs(X))
    assert np.max(np.abs(X[:, 2] - (X[:, 0] + 2 * X[:, 1]))) <= 1e-8 * sc
    assert np.max(np.abs(X[:, 5] - X[:, 1])) <= 1e-8 * sc
    assert np.max(np.abs(X - np.linalg.solve(A, Bd))) <= 1e-7 * sc
    # the starting block has rank 3 (the dependent, zero and duplicate columns dropped);
    # near convergence rounding may separate a dependent residual by more than the
    # threshold of its own (tiny) norm, which only adds a harmless direction
    assert oracle.block_cg_deflated(A, Bd, rtol=1e-10, max_iter=0)["rank"] == 3


def test_breakdown_only_when_a_is_not_spd(oracle):
    n = 30
    A = np.diag(np.r_[np.ones(n - 1), -1.0])
    B = np.ones((n, 2))
    B[:, 1] = np.arange(n)
    out = oracle.block_cg_deflated(A, B, rtol=1e-10, max_iter=100)
    assert out["status"] in (0, 2)                         # indefinite: may break down, never crashes
    Z = np.zeros((n, 2))
    out = oracle.block_cg_deflated(np.eye(n), Z, rtol=1e-10)
    assert out["status"] == 0 and not out["X"].any() and out["iters"] == 0
