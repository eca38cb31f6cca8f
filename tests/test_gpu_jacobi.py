"""GPU parity of the Jacobi iteration (ls_jacobi_solve) with the oracle.

Jacobi is a fixed linear recurrence, so after the same number of products
the GPU iterate and the oracle's differ only by the rounding of the products,
which the contraction (spectral radius below one) does not amplify: the
comparison after a fixed count is element by element.  To a tolerance, the
true relative residual (computed by the oracle) must reach rtol and the
product counts agree within one (the last test may fall either side of the
threshold).  Edge cases: n = 1, a diagonal matrix, b = 0, an exact initial
guess, a zero diagonal entry, the iteration limit, divergence, NaN input,
unsupported precision, both product modes, host buffers.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(ctx, gpu, A, b, x0=None, on_device=True, **kw):
    if on_device:
        Ad = torch.from_numpy(np.ascontiguousarray(A)).to(gpu)
        bd = torch.from_numpy(b).to(gpu)
        xd = torch.from_numpy(x0.copy() if x0 is not None else np.zeros(len(b))).to(gpu)
    else:
        Ad, bd = np.ascontiguousarray(A), b
        xd = x0.copy() if x0 is not None else np.zeros(len(b))
    o = B.make_opts(x0_given=int(x0 is not None), **kw)
    st, info = B.ls_jacobi_solve(ctx, Ad, bd, xd, o)
    x = xd.cpu().numpy() if on_device else xd
    return st, info, x


@pytest.mark.parametrize("n", [1, 2, 33, 257, 1000, 3001])
def test_jacobi_matches_oracle(ctx, gpu, oracle, n):
    A = inputs.nonsym_matrix(n, seed=600 + n)
    xs = inputs.solution(n, seed=600 + n)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    ref = oracle.jacobi(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    true_rel = np.linalg.norm(oracle.residual(A, b, x)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    assert abs(info["rel_res"] - true_rel) <= 1e-3 * true_rel + 1e-14   # A as the pair: 2^-48
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert info["launches"] >= 2 * info["iters"]


@pytest.mark.parametrize("f64_matvec", [0, 1])
@pytest.mark.parametrize("n", [100, 777, 2048])
def test_jacobi_fixed_count_elementwise(ctx, gpu, oracle, n, f64_matvec):
    A = inputs.nonsym_matrix(n, seed=700 + n)
    b = A @ inputs.solution(n, seed=700 + n)
    for k in (1, 2, 9):
        st, info, x = _solve(ctx, gpu, A, b, rtol=1e-300, max_iter=k, f64_matvec=f64_matvec)
        ref = oracle.jacobi(A, b, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert np.max(np.abs(x - ref["x"])) <= 1e-13 * np.max(np.abs(ref["x"])) + 1e-300
        assert info["rel_res"] == pytest.approx(ref["rel_res"], rel=1e-9)


def test_jacobi_host_buffers_determinism_initial_guess(ctx, gpu, oracle):
    n = 700
    A = inputs.nonsym_matrix(n, seed=9)
    xs = inputs.solution(n, seed=9)
    b = A @ xs
    st1, i1, x1 = _solve(ctx, gpu, A, b, rtol=1e-10)
    st2, i2, x2 = _solve(ctx, gpu, A, b, on_device=False, rtol=1e-10)
    st3, i3, x3 = _solve(ctx, gpu, A, b, rtol=1e-10)
    assert st1 == st2 == st3 == B.LS_OK
    assert i1["iters"] == i2["iters"] == i3["iters"]
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)
    x0 = xs + 1e-6 * inputs.solution(n, seed=11)
    st, info, x = _solve(ctx, gpu, A, b, x0=x0, rtol=1e-10)
    ref = oracle.jacobi(A, b, rtol=1e-10, x0=x0)
    assert st == B.LS_OK and info["iters"] < i1["iters"]
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    st, info, x = _solve(ctx, gpu, A, b, x0=xs.copy(), rtol=1e-10)
    assert st == B.LS_OK and info["iters"] == 1     # one product measures x0


def test_jacobi_edge_cases(ctx, gpu, oracle):
    d = np.array([2.0, -3.0, 0.5, 4.0])
    b = np.array([1.0, 2.0, 3.0, 4.0])
    st, info, x = _solve(ctx, gpu, np.diag(d), b, rtol=1e-14)
    assert st == B.LS_OK and info["iters"] == 2
    assert np.array_equal(x, b / d)
    n = 64
    A = inputs.nonsym_matrix(n, seed=2)
    st, info, x = _solve(ctx, gpu, A, np.zeros(n), x0=np.ones(n))
    assert st == B.LS_OK and not x.any() and info["iters"] == 0
    b = A @ inputs.solution(n, seed=2)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-14, max_iter=3)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 3
    Z = A.copy()
    Z[7, 7] = 0.0
    x0 = inputs.solution(n, seed=3)
    st, info, x = _solve(ctx, gpu, Z, b, x0=x0)
    ref = oracle.jacobi(Z, b, x0=x0)
    assert st == B.LS_BREAKDOWN == ref["status"]
    assert np.array_equal(x, x0)
    assert info["rel_res"] == pytest.approx(ref["rel_res"], rel=1e-12)
    S = inputs.spd_matrix(200, 0.01, seed=3)        # spectral radius of I - D^-1 A above one
    bs = S @ inputs.solution(200, seed=3)
    st, info, x = _solve(ctx, gpu, S, bs, max_iter=20)
    ref = oracle.jacobi(S, bs, max_iter=20)
    assert st == B.LS_NOT_CONVERGED == ref["status"]
    assert info["rel_res"] == pytest.approx(ref["rel_res"], rel=1e-6) and info["rel_res"] > 1.0
    bad = b.copy()
    bad[5] = np.nan
    st, info, x = _solve(ctx, gpu, A, bad)
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A, b, precision=B.LS_BF16_IR)
    assert st == B.LS_ERR_UNSUPPORTED


def test_jacobi_full_size(ctx, gpu, oracle):
    # the benchmark's size: the true residual, from the oracle, reaches rtol;
    # sampled rows of the last step checked one by one
    n = 16384
    A = inputs.nonsym_matrix(n, seed=17)
    b = A @ inputs.solution(n, seed=17)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    assert st == B.LS_OK
    r = oracle.residual(A, b, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    assert info["rel_res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-3)
