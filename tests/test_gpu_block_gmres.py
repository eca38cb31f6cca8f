"""GPU parity of restarted block GMRES (ls_block_gmres_solve) with the oracle.

The block iterate after k steps of a cycle is the least-squares minimiser
over the block Krylov space, unique whatever orthogonalisation builds the
basis (CholQR2 on the device, two-pass MGS in the oracle), so at a fixed
step count the comparison is element by element, across restarts too.  To a
tolerance: every column's true residual (computed by the oracle) reaches
rtol and the step counts agree within a few.  Edge cases: s = 1 (GMRES),
s = 16, n = 1, ragged n, slow convergence with restarts, an initial guess,
an exact initial guess, dependent columns (deflated by default, a breakdown
with deflate = 0), B = 0, the iteration limit, NaN input, unsupported options
and sizes, host buffers.

Deflation: a starting block with a dependent, a zero and a repeated column
has its dependent columns replaced by the same pseudo-random vectors on both
sides, so at a fixed step count the iterates agree element by element with
the oracle's; solved to rtol, every column reaches the LAPACK solution, the
dependent column's solution is the same combination of the others', the
zero column's is zero and the repeated column's equals the original's.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(ctx, gpu, A, Bm, X0=None, on_device=True, **kw):
    n, s = Bm.shape
    if on_device:
        Ad = torch.from_numpy(np.ascontiguousarray(A)).to(gpu)
        Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).to(gpu).t()
        Xd = torch.from_numpy(np.ascontiguousarray((X0 if X0 is not None else np.zeros((n, s))).T)).to(gpu).t()
    else:
        Ad, Bd = np.ascontiguousarray(A), np.asfortranarray(Bm)
        Xd = np.asfortranarray(X0.copy() if X0 is not None else np.zeros((n, s)))
    o = B.make_opts(x0_given=int(X0 is not None), **kw)
    st, info = B.ls_block_gmres_solve(ctx, Ad, Bd, Xd, o)
    X = Xd.cpu().numpy() if on_device else np.array(Xd)
    return st, info, X


def _true_rel(oracle, A, Bm, X):
    return max(np.linalg.norm(oracle.residual(A, Bm[:, j], X[:, j])) / np.linalg.norm(Bm[:, j])
               for j in range(Bm.shape[1]))


@pytest.mark.parametrize("n,s,m", [(1, 1, 3), (33, 1, 10), (257, 3, 8), (1000, 8, 10), (2049, 16, 8)])
def test_block_gmres_matches_oracle(ctx, gpu, oracle, n, s, m):
    A = inputs.nonsym_matrix(n, seed=110 + n)
    Bm = A @ inputs.solution(n, seed=111 + n, nrhs=s).reshape(n, s)
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-10, restart=m)
    ref = oracle.block_gmres(A, Bm, m=m, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    tr = _true_rel(oracle, A, Bm, X)
    assert tr <= 1e-10
    assert abs(info["rel_res"] - tr) <= 1e-3 * tr + 1e-14
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 10


@pytest.mark.parametrize("n,s,m", [(200, 4, 6), (513, 2, 5)])
def test_block_gmres_fixed_count_elementwise(ctx, gpu, oracle, n, s, m):
    A = inputs.restart_matrix(n, seed=120 + n)
    Bm = A @ inputs.solution(n, seed=121 + n, nrhs=s).reshape(n, s)
    for k in (1, 2, m - 1, m + 3):      # the last one crosses a restart
        st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-300, max_iter=k, restart=m)
        ref = oracle.block_gmres(A, Bm, m=m, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert info["outer_iters"] == ref["cycles"]
        assert np.max(np.abs(X - ref["X"])) <= 1e-10 * np.max(np.abs(ref["X"]))


def test_block_gmres_restarts_host_buffers_initial_guess(ctx, gpu, oracle):
    n, s, m = 600, 4, 5
    A = inputs.restart_matrix(n, seed=130)
    Xs = inputs.solution(n, seed=131, nrhs=s).reshape(n, s)
    Bm = A @ Xs
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-10, restart=m)
    ref = oracle.block_gmres(A, Bm, m=m, rtol=1e-10)
    assert st == B.LS_OK and info["outer_iters"] > 1 and _true_rel(oracle, A, Bm, X) <= 1e-10
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 10
    st2, info2, X2 = _solve(ctx, gpu, A, Bm, on_device=False, rtol=1e-10, restart=m)
    assert st2 == B.LS_OK and info2["iters"] == info["iters"] and np.array_equal(X, X2)
    st, info3, X = _solve(ctx, gpu, A, Bm, X0=Xs + 1e-6 * inputs.solution(n, seed=132, nrhs=s).reshape(n, s),
                          rtol=1e-10, restart=m)
    assert st == B.LS_OK and info3["iters"] < info["iters"] and _true_rel(oracle, A, Bm, X) <= 1e-10
    st, info4, X = _solve(ctx, gpu, A, Bm, X0=Xs.copy(), rtol=1e-10, restart=m)
    assert st == B.LS_OK and info4["iters"] == 0


def test_block_gmres_edge_cases(ctx, gpu):
    n = 64
    A = inputs.nonsym_matrix(n, seed=140)
    b = A @ inputs.solution(n, seed=140)
    st, info, X = _solve(ctx, gpu, A, np.stack([b, 2 * b], 1), restart=4, deflate=0)
    assert st == B.LS_BREAKDOWN
    st, info, X = _solve(ctx, gpu, A, np.stack([b, 2 * b], 1), restart=4)
    assert st == B.LS_OK and np.max(np.abs(X[:, 1] - 2 * X[:, 0])) <= 1e-8 * np.max(np.abs(X))
    st, info, X = _solve(ctx, gpu, A, np.zeros((n, 3)), restart=4)
    assert st == B.LS_OK and not X.any() and info["iters"] == 0
    Bm = A @ inputs.solution(n, seed=141, nrhs=3).reshape(n, 3)
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-300, max_iter=3, restart=2)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 3 and info["outer_iters"] == 2
    bad = Bm.copy()
    bad[3, 1] = np.nan
    st, info, X = _solve(ctx, gpu, A, bad, restart=4)
    assert st == B.LS_ERR_NAN
    for kw in (dict(precision=B.LS_BF16_IR), dict(f64_matvec=1)):
        st, info, X = _solve(ctx, gpu, A, Bm, restart=4, **kw)
        assert st == B.LS_ERR_UNSUPPORTED
    st, info, X = _solve(ctx, gpu, A, Bm, restart=100)        # 100 x 3 > 256
    assert st == B.LS_ERR_ARG


def _deficient_block(A, n, seed):
    """Columns b0, b1, b0 + 2 b1 (dependent), 0, b2, b1 (a repeat)."""
    Bf = A @ inputs.solution(n, seed=seed, nrhs=3).reshape(n, 3)
    return np.column_stack([Bf[:, 0], Bf[:, 1], Bf[:, 0] + 2 * Bf[:, 1], np.zeros(n), Bf[:, 2], Bf[:, 1]])


@pytest.mark.parametrize("n,m", [(200, 4), (777, 6)])
def test_block_gmres_deflated_fixed_count_elementwise(ctx, gpu, oracle, n, m):
    A = inputs.restart_matrix(n, seed=150 + n)
    Bm = _deficient_block(A, n, 151 + n)
    for k in (1, 2, m + 1):             # the last one crosses a restart
        st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-300, max_iter=k, restart=m)
        ref = oracle.block_gmres(A, Bm, m=m, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert info["outer_iters"] == ref["cycles"]
        assert np.max(np.abs(X - ref["X"])) <= 1e-10 * np.max(np.abs(ref["X"]))
        assert not X[:, 3].any()
        assert np.max(np.abs(X[:, 5] - X[:, 1])) <= 1e-13 * np.max(np.abs(X))


@pytest.mark.parametrize("n,m", [(300, 5), (1000, 10)])
def test_block_gmres_deflated_converges(ctx, gpu, oracle, n, m):
    A = inputs.nonsym_matrix(n, seed=160 + n)
    Bm = _deficient_block(A, n, 161 + n)
    st0, _, _ = _solve(ctx, gpu, A, Bm, rtol=1e-10, restart=m, deflate=0)
    assert st0 == B.LS_BREAKDOWN
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-10, restart=m)
    ref = oracle.block_gmres(A, Bm, m=m, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    cols = [0, 1, 2, 4, 5]
    tr = _true_rel(oracle, A, Bm[:, cols], X[:, cols])
    assert tr <= 1e-10 and abs(info["rel_res"] - tr) <= 1e-3 * tr + 1e-14
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 10
    sc = np.max(np.abs(X))
    assert not X[:, 3].any() and np.max(np.abs(X[:, 5] - X[:, 1])) <= 1e-12 * sc
    assert np.max(np.abs(X[:, 2] - (X[:, 0] + 2 * X[:, 1]))) <= 1e-8 * sc
    assert np.max(np.abs(X - np.linalg.solve(A, Bm))) <= 1e-7 * sc
    assert np.max(np.abs(X - ref["X"])) <= 1e-7 * sc
