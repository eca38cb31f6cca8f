"""GPU parity of forward Gauss-Seidel (ls_gauss_seidel_solve) with the oracle.

The device sweep is the oracle's in-place sweep written as a correction,
x(k+1) = x(k) + (D + L)^-1 (b - A x(k)), solved over 64-row blocks; after the
same number of sweeps the iterates differ only by rounding, which the
contraction does not amplify, so the fixed-count comparison is element by
element.  On a lower-triangular matrix one sweep is forward substitution
(checked against scipy at sizes that span many blocks and a ragged tail).
To a tolerance: the true relative residual (from the oracle) reaches rtol,
the counts agree within one.  Edge cases: n = 1, block-edge sizes, an SPD
matrix on which Jacobi diverges, b = 0, an exact initial guess, a zero
diagonal entry, the iteration limit, NaN input, unsupported precision, both
residual-product modes, host buffers and determinism.
"""
import numpy as np
import pytest
import scipy.linalg
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
    st, info = B.ls_gauss_seidel_solve(ctx, Ad, bd, xd, o)
    x = xd.cpu().numpy() if on_device else xd
    return st, info, x


@pytest.mark.parametrize("n", [1, 2, 33, 64, 65, 257, 1000, 3001])
def test_gs_matches_oracle(ctx, gpu, oracle, n):
    A = inputs.nonsym_matrix(n, seed=900 + n)
    b = A @ inputs.solution(n, seed=900 + n)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    ref = oracle.gauss_seidel(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    true_rel = np.linalg.norm(oracle.residual(A, b, x)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    assert abs(info["rel_res"] - true_rel) <= 1e-3 * true_rel + 1e-14   # A as the pair: 2^-48
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert info["launches"] >= 2 * info["iters"] - 1


@pytest.mark.parametrize("f64_matvec", [0, 1])
@pytest.mark.parametrize("n", [100, 777, 2048])
def test_gs_fixed_count_elementwise(ctx, gpu, oracle, n, f64_matvec):
    A = inputs.nonsym_matrix(n, seed=950 + n)
    b = A @ inputs.solution(n, seed=950 + n)
    for k in (1, 2, 6):
        st, info, x = _solve(ctx, gpu, A, b, rtol=1e-300, max_iter=k, f64_matvec=f64_matvec)
        ref = oracle.gauss_seidel(A, b, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert np.max(np.abs(x - ref["x"])) <= 1e-13 * np.max(np.abs(ref["x"])) + 1e-300
        assert info["rel_res"] == pytest.approx(ref["rel_res"], rel=1e-8)


@pytest.mark.parametrize("n", [64, 130, 1000, 4097])
def test_gs_lower_triangular_one_sweep(ctx, gpu, n):
    A = np.tril(inputs.nonsym_matrix(n, seed=31 + n))
    b = inputs.solution(n, seed=32 + n)
    # rtol above the rounding floor of a product with A as the pair (2^-48 a term)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-12)
    assert st == B.LS_OK and info["iters"] == 2
    ref = scipy.linalg.solve_triangular(A, b, lower=True)
    assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_gs_spd_where_jacobi_diverges(ctx, gpu, oracle):
    n = 300
    A = inputs.spd_matrix(n, 0.5, seed=4)
    b = A @ inputs.solution(n, seed=4)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    ref = oracle.gauss_seidel(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    assert abs(info["iters"] - ref["iters"]) <= 1 + ref["iters"] // 50
    stj, _ = B.ls_jacobi_solve(ctx, torch.from_numpy(A).to(gpu), torch.from_numpy(b).to(gpu),
                               torch.zeros(n, dtype=torch.float64, device=gpu),
                               B.make_opts(rtol=1e-10, max_iter=300))
    assert stj != B.LS_OK


def test_gs_host_buffers_determinism_initial_guess(ctx, gpu, oracle):
    n = 700
    A = inputs.nonsym_matrix(n, seed=19)
    xs = inputs.solution(n, seed=19)
    b = A @ xs
    st1, i1, x1 = _solve(ctx, gpu, A, b, rtol=1e-10)
    st2, i2, x2 = _solve(ctx, gpu, A, b, on_device=False, rtol=1e-10)
    st3, i3, x3 = _solve(ctx, gpu, A, b, rtol=1e-10)
    assert st1 == st2 == st3 == B.LS_OK
    assert i1["iters"] == i2["iters"] == i3["iters"]
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)
    x0 = xs + 1e-6 * inputs.solution(n, seed=21)
    st, info, x = _solve(ctx, gpu, A, b, x0=x0, rtol=1e-10)
    ref = oracle.gauss_seidel(A, b, rtol=1e-10, x0=x0)
    assert st == B.LS_OK and info["iters"] < i1["iters"]
    assert abs(info["iters"] - ref["iters"]) <= 1
    st, info, x = _solve(ctx, gpu, A, b, x0=xs.copy(), rtol=1e-10)
    assert st == B.LS_OK and info["iters"] == 1


def test_gs_edge_cases(ctx, gpu, oracle):
    n = 64
    A = inputs.nonsym_matrix(n, seed=2)
    st, info, x = _solve(ctx, gpu, A, np.zeros(n), x0=np.ones(n))
    assert st == B.LS_OK and not x.any() and info["iters"] == 0
    b = A @ inputs.solution(n, seed=2)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-300, max_iter=3)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 3
    Z = inputs.nonsym_matrix(150, seed=5)
    Z[100, 100] = 0.0
    bz = Z @ inputs.solution(150, seed=5)
    x0 = inputs.solution(150, seed=6)
    st, info, x = _solve(ctx, gpu, Z, bz, x0=x0)
    ref = oracle.gauss_seidel(Z, bz, x0=x0)
    assert st == B.LS_BREAKDOWN == ref["status"]
    assert np.array_equal(x, x0)
    assert info["rel_res"] == pytest.approx(ref["rel_res"], rel=1e-12)
    bad = b.copy()
    bad[5] = np.nan
    st, info, x = _solve(ctx, gpu, A, bad)
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A, b, precision=B.LS_BF16_IR)
    assert st == B.LS_ERR_UNSUPPORTED


def test_gs_full_size(ctx, gpu, oracle):
    # the benchmark's size: the true residual, from the oracle, reaches rtol
    n = 16384
    A = inputs.nonsym_matrix(n, seed=23)
    b = A @ inputs.solution(n, seed=23)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    assert st == B.LS_OK
    r = oracle.residual(A, b, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    assert info["rel_res"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-3)
