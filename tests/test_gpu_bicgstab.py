"""GPU parity of BiCGSTAB (ls_bicgstab_solve) with the oracle.

The solution is unique and the iterates differ from the oracle's only by
rounding order, so the comparison is by tolerance: the true relative residual
(computed by the oracle) must reach rtol, the error against the oracle's x
and against x* must stay within kappa * rtol (times a small safety factor),
and the product counts must agree within the slack that rounding gives a
non-minimising method.  Edge cases: n = 1, b = 0, an exact initial guess, a
forced breakdown, the iteration limit, NaN input, unsupported precision.
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
    st, info = B.ls_bicgstab_solve(ctx, Ad, bd, xd, o)
    x = xd.cpu().numpy() if on_device else xd
    return st, info, x


def _cond(A):
    s = np.linalg.svd(A, compute_uv=False)
    return s[0] / s[-1]


@pytest.mark.parametrize("n", [1, 2, 33, 257, 512, 1000, 3001])
def test_bicgstab_matches_oracle(ctx, gpu, oracle, n):
    A = inputs.nonsym_matrix(n, seed=400 + n)
    xs = inputs.solution(n, seed=400 + n)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    ref = oracle.bicgstab(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    true_rel = np.linalg.norm(oracle.residual(A, b, x)) / np.linalg.norm(b)
    assert true_rel <= 1e-10
    assert abs(info["true_rel_res"] - true_rel) <= 0.05 * true_rel + 1e-14
    kap = _cond(A)
    assert np.linalg.norm(x - ref["x"]) <= 4 * kap * 1e-10 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(x - xs) <= 4 * kap * 1e-10 * np.linalg.norm(xs)
    assert abs(info["iters"] - ref["iters"]) <= 4 + ref["iters"] // 10
    assert info["launches"] >= 2 * info["iters"]


@pytest.mark.parametrize("f64_matvec", [0, 1])
def test_bicgstab_both_matvec_modes_and_spd(ctx, gpu, oracle, f64_matvec):
    for A in (inputs.restart_matrix(600, seed=5), inputs.spd_matrix(600, 0.05, seed=5)):
        b = A @ inputs.solution(600, seed=6)
        st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10, f64_matvec=f64_matvec)
        assert st == B.LS_OK
        assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
        ref = oracle.bicgstab(A, b, rtol=1e-10)
        assert np.linalg.norm(x - ref["x"]) <= 4 * _cond(A) * 1e-10 * np.linalg.norm(ref["x"])


def test_bicgstab_host_buffers_and_determinism(ctx, gpu):
    n = 700
    A = inputs.nonsym_matrix(n, seed=9)
    b = A @ inputs.solution(n, seed=9)
    st1, i1, x1 = _solve(ctx, gpu, A, b, rtol=1e-10)
    st2, i2, x2 = _solve(ctx, gpu, A, b, on_device=False, rtol=1e-10)
    st3, i3, x3 = _solve(ctx, gpu, A, b, rtol=1e-10)
    assert st1 == st2 == st3 == B.LS_OK
    assert i1["iters"] == i2["iters"] == i3["iters"]
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)


def test_bicgstab_initial_guess(ctx, gpu, oracle):
    n = 300
    A = inputs.nonsym_matrix(n, seed=10)
    xs = inputs.solution(n, seed=10)
    b = A @ xs
    st, cold, _ = _solve(ctx, gpu, A, b, rtol=1e-10)
    x0 = xs + 1e-6 * inputs.solution(n, seed=11)
    st, info, x = _solve(ctx, gpu, A, b, x0=x0, rtol=1e-10)
    assert st == B.LS_OK and info["iters"] < cold["iters"]
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    st, info, x = _solve(ctx, gpu, A, b, x0=xs.copy(), rtol=1e-10)
    assert st == B.LS_OK and info["iters"] == 0


def test_bicgstab_edge_cases(ctx, gpu):
    n = 64
    A = inputs.nonsym_matrix(n, seed=2)
    st, info, x = _solve(ctx, gpu, A, np.zeros(n))
    assert st == B.LS_OK and not x.any() and info["iters"] == 0
    b = A @ inputs.solution(n, seed=2)
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-14, max_iter=3)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 3
    st, info, x = _solve(ctx, gpu, np.array([[0.0, 1.0], [-1.0, 0.0]]), np.array([1.0, 0.0]))
    assert st == B.LS_BREAKDOWN
    bad = b.copy()
    bad[5] = np.nan
    st, info, x = _solve(ctx, gpu, A, bad)
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A, b, precision=B.LS_BF16_IR)
    assert st == B.LS_ERR_UNSUPPORTED
