"""GPU parity of the FP64 conjugate gradient (ls_cg_solve) with the oracle.

The solution is unique, the iterates differ only by rounding order, so the
comparison is by tolerance: the true relative residual (computed by the
oracle) must reach rtol, the error against the oracle's x and against x* must
stay within kappa * rtol (times a small safety factor), and the iteration
counts must agree to within rounding (a couple of iterations).
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(ctx, gpu, A, b, x0=None, on_device=True, **kw):
    if on_device:
        Ad = torch.from_numpy(np.ascontiguousarray(A)).to(gpu) if isinstance(A, np.ndarray) else A
        bd = torch.from_numpy(b).to(gpu)
        xd = torch.from_numpy(x0.copy() if x0 is not None else np.zeros(len(b))).to(gpu)
    else:
        Ad, bd = A, b
        xd = x0.copy() if x0 is not None else np.zeros(len(b))
    o = B.make_opts(x0_given=int(x0 is not None), **kw)
    st, info = B.ls_cg_solve(ctx, Ad, bd, xd, o)
    x = xd.cpu().numpy() if on_device else xd
    return st, info, x


def _kappa(A):
    ev = np.linalg.eigvalsh(A)
    return ev[-1] / ev[0]


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("n,sigma", [(1, 0.1), (2, 0.1), (33, 0.1), (257, 0.1), (512, 0.1),
                                     (1000, 0.05), (3001, 0.1)])
def test_cg_matches_oracle(ctx, gpu, oracle, n, sigma, fused):
    """fused = 1: n <= 1000 runs as one kernel (A in shared memory), n = 3001
    on the general path; fused = 0: the general path throughout."""
    A = inputs.spd_matrix(n, sigma, seed=n)
    xs = inputs.solution(n, seed=n)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10, fused=fused)
    ref = oracle.cg(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    nb = np.linalg.norm(b)
    true_rel = np.linalg.norm(oracle.residual(A, b, x)) / nb
    assert true_rel <= 1e-10
    # the library's own true residual agrees (two summation orders: rounding noise)
    assert abs(info["true_rel_res"] - true_rel) <= 0.05 * true_rel + 1e-14
    kap = _kappa(A)
    assert np.linalg.norm(x - ref["x"]) <= 4 * kap * 1e-10 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(x - xs) <= 4 * kap * 1e-10 * np.linalg.norm(xs)
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 50
    if fused and n <= 1000:
        assert info["launches"] == 1
    else:
        assert info["launches"] >= 2 * info["iters"]


@pytest.mark.parametrize("n", [257, 1000])
def test_cg_native_fp64_matvec(ctx, gpu, oracle, n):
    """f64_matvec = 1 (FP64 FMA products) meets the same bar as the default
    double-single products, and the two agree within kappa * rtol."""
    A = inputs.spd_matrix(n, 0.05, seed=n + 5)
    xs = inputs.solution(n, seed=n + 5)
    b = A @ xs
    st1, i1, x1 = _solve(ctx, gpu, A, b, rtol=1e-10, f64_matvec=1)
    st0, i0, x0 = _solve(ctx, gpu, A, b, rtol=1e-10, f64_matvec=0)
    assert st0 == st1 == B.LS_OK
    for x in (x0, x1):
        assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    kap = _kappa(A)
    assert np.linalg.norm(x0 - x1) <= 4 * kap * 1e-10 * np.linalg.norm(xs)
    assert abs(i0["iters"] - i1["iters"]) <= 2


def test_cg_config_small_exact(ctx, gpu, oracle):
    """The n = 512, seed 0 SPD system (cond ~ 40): GPU and oracle agree."""
    n = 512
    A = inputs.spd_matrix(n, 0.1, seed=0)
    xs = inputs.solution(n, seed=0)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, rtol=1e-10)
    ref = oracle.cg(A, b, rtol=1e-10)
    assert st == B.LS_OK
    assert np.linalg.norm(x - ref["x"]) <= 1e-8 * np.linalg.norm(ref["x"])
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert abs(info["iters"] - ref["iters"]) <= 1


def test_cg_host_buffers_match_device(ctx, gpu):
    n = 640
    A = inputs.spd_matrix(n, 0.1, seed=4)
    b = A @ inputs.solution(n, seed=4)
    st1, i1, x1 = _solve(ctx, gpu, A, b, rtol=1e-11)
    st2, i2, x2 = _solve(ctx, gpu, A, b, rtol=1e-11, on_device=False)
    assert st1 == st2 == B.LS_OK
    assert i1["iters"] == i2["iters"]
    assert np.array_equal(x1, x2)        # same kernels on the same bits


def test_cg_deterministic(ctx, gpu):
    n = 1500
    A = inputs.spd_matrix(n, 0.01, seed=5)
    b = A @ inputs.solution(n, seed=5)
    _, i1, x1 = _solve(ctx, gpu, A, b)
    _, i2, x2 = _solve(ctx, gpu, A, b)
    assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)


def test_cg_padded_and_odd_lda(ctx, gpu, oracle):
    n = 333
    A = inputs.spd_matrix(n, 0.1, seed=6)
    b = A @ inputs.solution(n, seed=6)
    for pad in (3, 64):                 # odd lda: plain-load GEMV; aligned: TMA
        full = np.zeros((n, n + pad))
        full[:, :n] = A
        Ad = torch.from_numpy(full).to(gpu)[:, :n]
        st, info, x = _solve(ctx, gpu, Ad, b)
        assert st == B.LS_OK
        assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)


def test_cg_initial_guess(ctx, gpu, oracle):
    n = 400
    A = inputs.spd_matrix(n, 0.1, seed=7)
    xs = inputs.solution(n, seed=7)
    b = A @ xs
    x0 = xs + 1e-6 * inputs.solution(n, seed=8)
    st, info, x = _solve(ctx, gpu, A, b, x0=x0)
    _, cold, _ = _solve(ctx, gpu, A, b)
    assert st == B.LS_OK and info["iters"] < cold["iters"]
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    # exact start: no iteration at all
    st, info, x = _solve(ctx, gpu, np.eye(n) * 2.0, 2.0 * xs, x0=xs)
    assert st == B.LS_OK and info["iters"] == 0 and np.array_equal(x, xs)


@pytest.mark.parametrize("fused", [0, 1])
def test_cg_edge_cases(ctx, gpu, fused):
    n = 200
    A = inputs.spd_matrix(n, 0.1, seed=9)
    xs = inputs.solution(n, seed=9)
    # b = 0 -> x = 0 (also when an initial guess is given)
    st, info, x = _solve(ctx, gpu, A, np.zeros(n), x0=xs, fused=fused)
    assert st == B.LS_OK and not x.any() and info["iters"] == 0
    # iteration limit
    st, info, x = _solve(ctx, gpu, A, A @ xs, rtol=1e-14, max_iter=3, fused=fused)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 3
    # negative definite: breakdown, reported not crashed
    st, info, x = _solve(ctx, gpu, -A, A @ xs, fused=fused)
    assert st == B.LS_BREAKDOWN
    # NaN in b
    b = A @ xs
    b[5] = np.nan
    st, info, x = _solve(ctx, gpu, A, b, fused=fused)
    assert st == B.LS_ERR_NAN
    # the context is still healthy afterwards
    st, info, x = _solve(ctx, gpu, A, A @ xs, fused=fused)
    assert st == B.LS_OK
    # bad arguments
    xd = torch.zeros(n, dtype=torch.float64, device=gpu)
    assert B.load().ls_cg_solve(ctx, -1, None, 0, None, None, None, None) == B.LS_ERR_ARG
    assert B.ls_cg_solve(ctx, torch.zeros((n, n), dtype=torch.float64, device=gpu),
                         xd, xd, B.make_opts(rtol=-1.0))[0] == B.LS_ERR_ARG
