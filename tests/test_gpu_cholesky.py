"""GPU parity of the Cholesky method (ls_chol_factor, ls_chol_solve) with the
oracle.

The factorization is the oracle's column factorization step for step (IEEE
square root and division, multiply and subtract unfused, each element's
updates in step order), with b carried as an extra row, so L and y = L^-1 b
are compared bit for bit.  The back substitution sums in another order, so x
is compared with the oracle's x within a few units of rounding of the solve:
|x - x_ref| <= 64 n kappa 2^-52 max|x_ref| (as for the LU).  Edge cases:
n = 1, 2, panel borders (31, 32, 33, 64, 65), ragged sizes, a matrix that is
not positive definite (the failing step is reported), a zero pivot, NaN
input, only the lower triangle read, unsupported precision, host buffers,
n = 0.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _factor(ctx, gpu, A, b):
    n = A.shape[0]
    L = torch.full((n, n), np.nan, dtype=torch.float64, device=gpu)
    y = torch.full((n,), np.nan, dtype=torch.float64, device=gpu)
    st, step = B.ls_chol_factor(ctx, torch.from_numpy(np.ascontiguousarray(A)).to(gpu),
                                torch.from_numpy(b).to(gpu), L, y)
    return st, step, L.cpu().numpy(), y.cpu().numpy()


def _solve(ctx, gpu, A, b, on_device=True, **kw):
    if on_device:
        x = torch.zeros(len(b), dtype=torch.float64, device=gpu)
        st, info = B.ls_chol_solve(ctx, torch.from_numpy(np.ascontiguousarray(A)).to(gpu),
                                   torch.from_numpy(b).to(gpu), x, B.make_opts(**kw))
        return st, info, x.cpu().numpy()
    x = np.zeros(len(b))
    st, info = B.ls_chol_solve(ctx, np.ascontiguousarray(A), b, x, B.make_opts(**kw))
    return st, info, x


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 64, 65, 257, 1000, 2049])
def test_cholesky_factor_bit_exact(ctx, gpu, oracle, n):
    A = inputs.spd_matrix(n, 0.1, seed=190 + n)
    b = A @ inputs.solution(n, seed=191 + n)
    st, step, L, y = _factor(ctx, gpu, A, b)
    Lr, str_ = oracle.chol_factor(A)
    assert st == B.LS_OK == str_ and step == -1
    assert np.array_equal(L, Lr)
    assert np.array_equal(y, oracle.chol_forward(Lr, b))


def test_cholesky_reads_only_the_lower_triangle(ctx, gpu, oracle):
    n = 150
    A = inputs.spd_matrix(n, 0.05, seed=200)
    b = A @ inputs.solution(n, seed=201)
    Ag = A.copy()
    Ag[np.triu_indices(n, 1)] = np.nan                      # never read
    st, _, L, y = _factor(ctx, gpu, Ag, b)
    Lr, _ = oracle.chol_factor(A)
    assert st == B.LS_OK and np.array_equal(L, Lr) and np.array_equal(y, oracle.chol_forward(Lr, b))


@pytest.mark.parametrize("n,sigma", [(1, 0.1), (50, 0.1), (777, 0.05), (3001, 0.1), (2000, 1e-3)])
def test_cholesky_solve_matches_oracle(ctx, gpu, oracle, n, sigma):
    A = inputs.spd_matrix(n, sigma, seed=210 + n)
    xs = inputs.solution(n, seed=211 + n)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b)
    xr, str_ = oracle.chol_solve(A, b)
    assert st == B.LS_OK == str_
    ev = np.linalg.eigvalsh(A)
    kap = ev[-1] / ev[0]
    assert np.max(np.abs(x - xr)) <= 64 * n * kap * 2.0 ** -52 * np.max(np.abs(xr))
    r = oracle.residual(A, b, x)
    assert info["true_rel_res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-6, abs=1e-14)
    assert info["true_rel_res"] <= 1e-10
    assert info["iters"] == 0 and info["launches"] > 0


def test_cholesky_edge_cases(ctx, gpu, oracle):
    n = 70
    A = inputs.spd_matrix(n, 0.1, seed=220)
    b = A @ inputs.solution(n, seed=221)
    # not positive definite: the pivot of step 40 is negative
    Ab = np.eye(n)
    Ab[40, 40] = -1.0
    st, step, L, y = _factor(ctx, gpu, Ab, np.ones(n))
    assert st == B.LS_BREAKDOWN == oracle.chol_factor(Ab)[1] and step == 40
    st, info, x = _solve(ctx, gpu, Ab, np.ones(n))
    assert st == B.LS_BREAKDOWN and not x.any()
    Z = A.copy()
    Z[5, :] = Z[:, 5] = 0.0                                 # a zero pivot at step 5
    st, step, _, _ = _factor(ctx, gpu, Z, b)
    assert st == B.LS_BREAKDOWN and step == 5
    bad = b.copy()
    bad[3] = np.nan
    st, info, x = _solve(ctx, gpu, A, bad)
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A, b, precision=B.LS_BF16_IR)
    assert st == B.LS_ERR_UNSUPPORTED
    st1, _, x1 = _solve(ctx, gpu, A, b)
    st2, _, x2 = _solve(ctx, gpu, A, b, on_device=False)
    assert st1 == st2 == B.LS_OK and np.array_equal(x1, x2)
    e = np.zeros(0)
    assert B.load().ls_chol_solve(ctx, 0, None, 0, None, None, None, None) == B.LS_OK
