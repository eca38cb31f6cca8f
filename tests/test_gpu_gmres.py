"""GPU parity of restarted GMRES(m) (ls_gmres_solve) with the oracle.

The GPU uses classical Gram-Schmidt with a conditional second pass; the
oracle uses modified Gram-Schmidt.  Both are exact-arithmetic GMRES, so the
comparison is by tolerance on the solution and the true residual, and
iteration counts must agree within a few steps.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(ctx, gpu, A, b, x0=None, **kw):
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(gpu)
    bd = torch.from_numpy(b).to(gpu)
    xd = torch.from_numpy(x0.copy() if x0 is not None else np.zeros(len(b))).to(gpu)
    o = B.make_opts(x0_given=int(x0 is not None), **kw)
    st, info = B.ls_gmres_solve(ctx, Ad, bd, xd, o)
    return st, info, xd.cpu().numpy()


def _cond(A):
    s = np.linalg.svd(A, compute_uv=False)
    return s[0] / s[-1]


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("n,m", [(1, 30), (2, 30), (33, 30), (257, 30), (512, 30), (1000, 50),
                                 (3001, 30)])
def test_gmres_matches_oracle(ctx, gpu, oracle, n, m, fused):
    A = inputs.nonsym_matrix(n, seed=n)
    xs = inputs.solution(n, seed=n)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, restart=m, rtol=1e-10, fused=fused)
    ref = oracle.gmres(A, b, m=m, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    true_rel = np.linalg.norm(oracle.residual(A, b, x)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    kap = _cond(A)
    assert np.linalg.norm(x - ref["x"]) <= 4 * kap * 1e-10 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(x - xs) <= 4 * kap * 1e-10 * np.linalg.norm(xs)
    assert abs(info["iters"] - ref["iters"]) <= 1


@pytest.mark.parametrize("f64_matvec", [0, 1])
def test_gmres_both_matvec_modes(ctx, gpu, oracle, f64_matvec):
    n = 700
    A = inputs.nonsym_matrix(n, seed=77)
    xs = inputs.solution(n, seed=77)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, restart=30, rtol=1e-10, f64_matvec=f64_matvec)
    ref = oracle.gmres(A, b, m=30, rtol=1e-10)
    assert st == B.LS_OK
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    assert abs(info["iters"] - ref["iters"]) <= 1


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("m,reorth", [(5, 0), (12, 1), (30, 0)])
def test_gmres_restarts(ctx, gpu, oracle, m, reorth, fused):
    n = 300
    A = inputs.restart_matrix(n, seed=10)
    b = A @ inputs.solution(n, seed=10)
    st, info, x = _solve(ctx, gpu, A, b, restart=m, rtol=1e-10, reorth=reorth, max_iter=20000,
                         fused=fused)
    ref = oracle.gmres(A, b, m=m, rtol=1e-10, max_iter=20000)
    assert st == B.LS_OK == ref["status"]
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    assert info["outer_iters"] >= 2
    assert abs(info["iters"] - ref["iters"]) <= 0.1 * ref["iters"] + 3


@pytest.mark.parametrize("fused", [0, 1])
def test_gmres_first_cycle_is_minimal_residual(ctx, gpu, oracle, fused):
    """k steps of one cycle: same iterate as the oracle's (both are the
    unique minimiser of ||b - A x|| over K_k)."""
    n = 200
    A = inputs.restart_matrix(n, seed=11)
    b = A @ inputs.solution(n, seed=11)
    for k in (1, 3, 8):
        st, info, x = _solve(ctx, gpu, A, b, restart=30, rtol=0.0, max_iter=k, fused=fused)
        ref = oracle.gmres(A, b, m=30, rtol=0.0, max_iter=k)
        assert st == B.LS_NOT_CONVERGED and info["iters"] == k
        assert np.linalg.norm(x - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("fused", [0, 1])
def test_gmres_edge_cases(ctx, gpu, oracle, fused):
    n = 64
    xs = inputs.solution(n, seed=12)
    st, info, x = _solve(ctx, gpu, 2.0 * np.eye(n), 2.0 * xs, restart=10, fused=fused)
    assert st == B.LS_OK and info["iters"] == 1
    assert np.allclose(x, xs, rtol=0, atol=1e-15)
    A = inputs.nonsym_matrix(n, seed=12)
    st, info, x = _solve(ctx, gpu, A, np.zeros(n), x0=xs, fused=fused)
    assert st == B.LS_OK and not x.any()
    st, info, x = _solve(ctx, gpu, A, A @ xs, x0=xs + 1e-9, fused=fused)
    assert st == B.LS_OK and info["iters"] <= 3
    b = A @ xs
    b[0] = np.inf
    st, info, x = _solve(ctx, gpu, A, b, fused=fused)
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A, A @ xs, restart=0, fused=fused)
    assert st == B.LS_ERR_ARG
    st, info, x = _solve(ctx, gpu, A, A @ xs, restart=B.LS_MAX_RESTART + 1, fused=fused)
    assert st == B.LS_ERR_ARG
    # singular system with b outside the range: not a false success
    S = np.diag(np.r_[0.0, np.ones(n - 1)])
    st, info, x = _solve(ctx, gpu, S, np.ones(n), restart=4, max_iter=40, fused=fused)
    assert st in (B.LS_BREAKDOWN, B.LS_NOT_CONVERGED)
    st, info, x = _solve(ctx, gpu, A, A @ xs, restart=30, fused=fused)
    assert st == B.LS_OK
