"""Pins for the oracle's restarted block GMRES (CPU only).

Independent checks: after k block steps of the first cycle the iterate is the
least-squares minimiser of ||B - A X||_F over X_0 + K_k(A, R_0), the block
Krylov space (numpy: explicit basis, lstsq); with s = 1 it is the oracle's
GMRES (itself pinned); with n = s m' it terminates within m' block steps;
restarted runs reach the LAPACK solution; without deflation a rank-deficient
right-hand side block breaks down.

Deflation (the default): the vectors that replace dependent columns are
SplitMix64's published outputs scaled to [-1, 1); after k block steps from a
rank-deficient block the iterate is the least-squares minimiser over
X_0 + K_k(A, [R_kept, Z]) (numpy: explicit basis from the kept columns and
the replacements, lstsq); blocks with a zero, a repeated or a dependent
column reach the LAPACK solution, the dependent column's solution being the
same combination of the others' (linearity) and the zero column's zero; on a
full-rank block deflation changes nothing, bit for bit.
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
    assert oracle.block_gmres(A, np.stack([b, 2 * b], 1), m=5, deflate=0)["status"] == oracle.BREAKDOWN
    B = A @ inputs.solution(n, seed=10, nrhs=3)
    out = oracle.block_gmres(A, B, m=2, rtol=1e-300, max_iter=3)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 3 and out["cycles"] == 2
    out = oracle.block_gmres(A, np.zeros((n, 2)), m=3)
    assert out["status"] == oracle.OK and out["iters"] == 0 and not out["X"].any()


# SplitMix64 seeded with 0: its first three outputs as published
SPLITMIX64_SEED0 = (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F)


def _splitmix64(k):
    """Output k (from 0) of SplitMix64 seeded with 0, restated in Python."""
    m = (1 << 64) - 1
    x = ((k + 1) * 0x9E3779B97F4A7C15) & m
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & m
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & m
    return x ^ (x >> 31)


def _replacement(n, c):
    return np.array([2.0 * ((_splitmix64((c << 32) | i) >> 11) * 2.0 ** -53) - 1.0 for i in range(n)])


def test_replacement_vectors_are_splitmix64(oracle):
    assert tuple(_splitmix64(k) for k in range(3)) == SPLITMIX64_SEED0
    z = oracle.block_gmres_replacement(3, 0)
    assert np.array_equal(z, [2.0 * ((v >> 11) * 2.0 ** -53) - 1.0 for v in SPLITMIX64_SEED0])
    for n, c in ((1, 0), (50, 1), (33, 7)):
        assert np.array_equal(oracle.block_gmres_replacement(n, c), _replacement(n, c))
    assert not np.array_equal(oracle.block_gmres_replacement(40, 2), oracle.block_gmres_replacement(40, 3))


def _deficient_block(A, n, seed):
    """Columns b0, b1, b0 + 2 b1 (dependent), 0, b2, b1 (a duplicate)."""
    Bf = A @ inputs.solution(n, seed=seed, nrhs=3)
    return np.column_stack([Bf[:, 0], Bf[:, 1], Bf[:, 0] + 2 * Bf[:, 1], np.zeros(n), Bf[:, 2], Bf[:, 1]])


@pytest.mark.parametrize("k", [1, 2, 4])
def test_deflated_block_gmres_minimises_over_kept_and_replacement_directions(oracle, k):
    n = 60
    A = inputs.restart_matrix(n, seed=23)
    Bd = _deficient_block(A, n, 24)
    dead = (2, 3, 5)
    out = oracle.block_gmres(A, Bd, m=6, rtol=1e-300, max_iter=k)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == k and out["cycles"] == 1
    start = Bd.copy()
    for c in dead:
        start[:, c] = _replacement(n, c)
    blocks = [start]
    for _ in range(k - 1):
        blocks.append(A @ blocks[-1])
    V = np.linalg.qr(np.hstack(blocks))[0]
    ref = np.linalg.lstsq(A @ V, Bd, rcond=None)[0]
    ref = V @ ref
    assert np.max(np.abs(out["X"] - ref)) <= 1e-9 * np.max(np.abs(ref))
    # without the replacements the space is smaller: the residual is not below the minimiser's
    kept = np.delete(start, dead, axis=1)
    blocks = [kept]
    for _ in range(k - 1):
        blocks.append(A @ blocks[-1])
    W = np.linalg.qr(np.hstack(blocks))[0]
    small = W @ np.linalg.lstsq(A @ W, Bd, rcond=None)[0]
    assert np.linalg.norm(Bd - A @ out["X"]) <= np.linalg.norm(Bd - A @ small) * (1 + 1e-9)


@pytest.mark.parametrize("m", [3, 8])
def test_deflated_block_gmres_rank_deficient_blocks_converge(oracle, m):
    n = 90
    A = inputs.nonsym_matrix(n, seed=25)
    Bd = _deficient_block(A, n, 26)
    assert oracle.block_gmres(A, Bd, m=m, rtol=1e-10, deflate=0)["status"] == oracle.BREAKDOWN
    out = oracle.block_gmres(A, Bd, m=m, rtol=1e-10)
    assert out["status"] == oracle.OK and out["rel_res"] <= 1e-10
    X = out["X"]
    assert not X[:, 3].any()                               # b = 0 -> x = 0
    sc = np.max(np.abs(X))
    assert np.max(np.abs(X[:, 2] - (X[:, 0] + 2 * X[:, 1]))) <= 1e-8 * sc
    assert np.max(np.abs(X[:, 5] - X[:, 1])) <= 1e-8 * sc
    assert np.max(np.abs(X - np.linalg.solve(A, Bd))) <= 1e-7 * sc


def test_deflation_changes_nothing_on_a_full_rank_block(oracle):
    n, s = 80, 4
    A = inputs.restart_matrix(n, seed=27)
    B = A @ inputs.solution(n, seed=28, nrhs=s)
    for k in (2, 9):
        a = oracle.block_gmres(A, B, m=5, rtol=1e-300, max_iter=k, deflate=1)
        b = oracle.block_gmres(A, B, m=5, rtol=1e-300, max_iter=k, deflate=0)
        assert np.array_equal(a["X"], b["X"]) and a["cycles"] == b["cycles"] == (k + 4) // 5
