"""GPU parity of the direct method (ls_lu_factor, ls_lu_solve) with the oracle.

The elimination is the oracle's step for step (same pivot rule, IEEE division,
multiply and subtract unfused), so the factors, the pivot rows and
y = L^-1 P b are compared bit for bit; the back substitution sums in another
order, so x is compared to within a few units of rounding of the solve.
Edge cases: n = 1, 2, ragged sizes, pivoting with ties (integer matrices),
a singular matrix (zero pivot), NaN input, unsupported precision, host
buffers.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _factor(ctx, gpu, A, b):
    n = A.shape[0]
    LU = torch.zeros((n, n), dtype=torch.float64, device=gpu)
    ipiv = torch.zeros(n, dtype=torch.int32, device=gpu)
    y = torch.zeros(n, dtype=torch.float64, device=gpu)
    st = B.ls_lu_factor(ctx, torch.from_numpy(np.ascontiguousarray(A)).to(gpu), torch.from_numpy(b).to(gpu),
                        LU, ipiv, y)
    return st, LU.cpu().numpy(), ipiv.cpu().numpy(), y.cpu().numpy()


def _solve(ctx, gpu, A, b, on_device=True, **kw):
    if on_device:
        x = torch.zeros(len(b), dtype=torch.float64, device=gpu)
        st, info = B.ls_lu_solve(ctx, torch.from_numpy(np.ascontiguousarray(A)).to(gpu),
                                 torch.from_numpy(b).to(gpu), x, B.make_opts(**kw))
        return st, info, x.cpu().numpy()
    x = np.zeros(len(b))
    st, info = B.ls_lu_solve(ctx, np.ascontiguousarray(A), b, x, B.make_opts(**kw))
    return st, info, x


@pytest.mark.parametrize("n", [1, 2, 33, 257, 1000, 2049])
def test_lu_factor_bit_exact(ctx, gpu, oracle, n):
    A = inputs.nonsym_matrix(n, seed=160 + n, shift=0.0, scale=1.0)     # pivoting matters
    b = A @ inputs.solution(n, seed=161 + n)
    st, LU, ipiv, y = _factor(ctx, gpu, A, b)
    LUr, ipr, yr, str_ = oracle.ge_factor(A, b)
    assert st == B.LS_OK == str_
    assert np.array_equal(ipiv, ipr)
    assert np.array_equal(LU, LUr)
    assert np.array_equal(y, yr)


def test_lu_factor_ties_first_row(ctx, gpu, oracle):
    rng = np.random.default_rng(5)
    A = rng.integers(-3, 4, size=(120, 120)).astype(np.float64)   # many equal |a|
    A += 8 * np.eye(120) * (rng.random(120) < 0.3)
    b = rng.integers(-5, 6, size=120).astype(np.float64)
    st, LU, ipiv, y = _factor(ctx, gpu, A, b)
    LUr, ipr, yr, str_ = oracle.ge_factor(A, b)
    assert st == str_
    assert np.array_equal(ipiv, ipr) and np.array_equal(LU, LUr) and np.array_equal(y, yr)


@pytest.mark.parametrize("n", [1, 50, 777, 3001])
def test_lu_solve_matches_oracle(ctx, gpu, oracle, n):
    A = inputs.nonsym_matrix(n, seed=170 + n, shift=0.0, scale=1.0)
    xs = inputs.solution(n, seed=171 + n)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b)
    xr, str_ = oracle.ge_solve(A, b)
    assert st == B.LS_OK == str_
    kap = np.linalg.cond(A)
    assert np.max(np.abs(x - xr)) <= 64 * n * kap * 2.0 ** -52 * np.max(np.abs(xr))
    r = oracle.residual(A, b, x)
    # residual norms at the rounding floor differ by their own rounding
    assert info["true_rel_res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-6, abs=1e-14)
    assert info["true_rel_res"] <= 1e-10
    assert info["iters"] == 0 and info["launches"] > 0


def test_lu_edge_cases(ctx, gpu, oracle):
    n = 40
    A = inputs.nonsym_matrix(n, seed=180, shift=0.0, scale=1.0)
    A[:, 7] = 0.0                                           # singular: a zero pivot at step 7
    b = np.ones(n)
    st, info, x = _solve(ctx, gpu, A, b)
    assert st == B.LS_BREAKDOWN == oracle.ge_solve(A, b)[1]
    assert not x.any()
    A2 = inputs.nonsym_matrix(n, seed=181)
    b2 = A2 @ inputs.solution(n, seed=181)
    bad = b2.copy()
    bad[3] = np.nan
    st, info, x = _solve(ctx, gpu, A2, bad)
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A2, b2, precision=B.LS_BF16_IR)
    assert st == B.LS_ERR_UNSUPPORTED
    st1, _, x1 = _solve(ctx, gpu, A2, b2)
    st2, _, x2 = _solve(ctx, gpu, A2, b2, on_device=False)
    assert st1 == st2 == B.LS_OK and np.array_equal(x1, x2)
