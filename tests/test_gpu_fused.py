"""GPU parity of the fused small-system solvers: a CG or GMRES(m) solve as one
persistent kernel with A's rows kept in shared memory (ls_opts.fused = 1,
taken when the rows fit; n up to about 1800 on 152 SMs).  Up to n of about
650 the CTAs form one thread-block cluster (distributed shared memory);
above, or with LS_FUSED_CTAS set, a cooperative grid communicating through
global memory.

The iteration is the general path's, so the same bars apply:
* after k steps the iterate is the oracle's up to rounding, element by element:
  |x - x_oracle|_max <= k kappa sqrt(n) 2^-48 |x_oracle|_max (A carried to
  2^-48 by the FP32 pair, sums rounding at 2^-53);
* converged solves reach the tolerance on the true residual (computed by the
  oracle) and agree with the oracle's x within ||A^-1|| (||r|| + ||r_oracle||);
* iteration counts agree with the oracle's and with the general path's to
  within rounding;
* one launch per solve (the general path takes two or more per step).
Ragged sizes (n not a multiple of the 8 rows per CTA or of the 4-column
vectors) and other CTA counts (LS_FUSED_CTAS) are covered.
"""
import math
import os

import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu

U48 = 2.0 ** -48


def _run(fn, ctx, gpu, A, b, x0=None, **kw):
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(gpu) if isinstance(A, np.ndarray) else A
    bd = torch.from_numpy(b).to(gpu)
    xd = torch.from_numpy(x0.copy() if x0 is not None else np.zeros(len(b))).to(gpu)
    st, info = fn(ctx, Ad, bd, xd, B.make_opts(x0_given=int(x0 is not None), **kw))
    return st, info, xd.cpu().numpy()


def _cg(ctx, gpu, A, b, **kw):
    return _run(B.ls_cg_solve, ctx, gpu, A, b, **kw)


def _gmres(ctx, gpu, A, b, **kw):
    return _run(B.ls_gmres_solve, ctx, gpu, A, b, **kw)


def _spd_kappa(A):
    ev = np.linalg.eigvalsh(A)
    return ev[-1] / ev[0], 1.0 / ev[0]


def _svd_kappa(A):
    s = np.linalg.svd(A, compute_uv=False)
    return s[0] / s[-1], 1.0 / s[-1]


def _converged_ok(oracle, A, b, x, xref, inv_norm, rtol):
    """x - xref = A^-1 (r_ref - r), so |x - xref| <= ||A^-1|| (||r|| + ||r_ref||),
    plus the rounding of the two computed residuals (gamma_{n+1} (|b| + |A||x|)
    each)."""
    rg = np.linalg.norm(oracle.residual(A, b, x))
    ro = np.linalg.norm(oracle.residual(A, b, xref))
    assert rg <= rtol * np.linalg.norm(b)
    n = len(b)
    ev = (n + 1) * 2.0 ** -53 * (np.linalg.norm(b) + np.linalg.norm(np.abs(A) @ np.abs(xref)))
    assert np.max(np.abs(x - xref)) <= inv_norm * (rg + ro + 2 * ev)


# ---------------------------------------------------------------------------
# converged solves against the oracle, ragged sizes, one launch each
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 7, 13, 129, 512, 1001, 1800])
def test_cg_fused_matches_oracle(ctx, gpu, oracle, n):
    A = inputs.spd_matrix(n, 0.1, seed=40 + n)
    b = A @ inputs.solution(n, seed=41 + n)
    st, info, x = _cg(ctx, gpu, A, b, rtol=1e-10)
    ref = oracle.cg(A, b, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    assert info["launches"] == 1
    _, inv = _spd_kappa(A)
    _converged_ok(oracle, A, b, x, ref["x"], inv, 1e-10)
    assert abs(info["iters"] - ref["iters"]) <= 1 + ref["iters"] // 50
    assert abs(info["true_rel_res"] - np.linalg.norm(oracle.residual(A, b, x)) / np.linalg.norm(b)) \
        <= 0.05 * info["true_rel_res"] + 1e-14


@pytest.mark.parametrize("n,m", [(1, 30), (2, 30), (3, 5), (13, 30), (129, 30), (512, 30), (1001, 50),
                                 (1800, 30)])
def test_gmres_fused_matches_oracle(ctx, gpu, oracle, n, m):
    A = inputs.nonsym_matrix(n, seed=50 + n)
    b = A @ inputs.solution(n, seed=51 + n)
    st, info, x = _gmres(ctx, gpu, A, b, restart=m, rtol=1e-10)
    ref = oracle.gmres(A, b, m=m, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    assert info["launches"] == 1
    _, inv = _svd_kappa(A)
    _converged_ok(oracle, A, b, x, ref["x"], inv, 1e-10)
    assert abs(info["iters"] - ref["iters"]) <= 1
    # the reported estimate is the last step's residual estimate (0 only for an exact solve)
    assert 0.0 <= info["rel_res"] <= 1e-10
    if n >= 13:
        assert info["rel_res"] > 0.0


# ---------------------------------------------------------------------------
# fixed step counts, element by element, in several CTA shapes
# ---------------------------------------------------------------------------
@pytest.fixture
def ctas():
    old = os.environ.get("LS_FUSED_CTAS")
    yield
    if old is None:
        os.environ.pop("LS_FUSED_CTAS", None)
    else:
        os.environ["LS_FUSED_CTAS"] = old


@pytest.mark.parametrize("n,G", [(512, 0), (512, 64), (997, 0), (150, 5), (997, 64), (997, 152)])
def test_cg_fused_fixed_count_elementwise(ctx, gpu, oracle, ctas, n, G):
    """G = 0: the default shape (n = 512: one cluster of 16 CTAs; n = 997: the
    global form, 8 rows per CTA); otherwise the global form with G CTAs."""
    if G:
        os.environ["LS_FUSED_CTAS"] = str(G)
    A = inputs.spd_matrix(n, 0.1, seed=60)
    b = A @ inputs.solution(n, seed=61)
    kappa, _ = _spd_kappa(A)
    for k in (1, 2, 5, 20):
        st, info, x = _cg(ctx, gpu, A, b, rtol=1e-300, max_iter=k)
        ref = oracle.cg(A, b, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k and info["launches"] == 1
        tol = k * kappa * math.sqrt(n) * U48 * np.max(np.abs(ref["x"]))
        assert np.max(np.abs(x - ref["x"])) <= tol, (G, k)


@pytest.mark.parametrize("n,G,reorth", [(512, 0, 0), (512, 0, 1), (512, 64, 0), (901, 0, 0), (150, 5, 1),
                                         (901, 152, 0)])
def test_gmres_fused_fixed_count_elementwise(ctx, gpu, oracle, ctas, n, G, reorth):
    """k < m: the first cycle; k > m: across restarts (m = 8)."""
    m = 8
    if G:
        os.environ["LS_FUSED_CTAS"] = str(G)
    A = inputs.restart_matrix(n, seed=62)
    b = A @ inputs.solution(n, seed=63)
    kappa, _ = _svd_kappa(A)
    for k in (1, 2, 5, 8, 11, 20):
        st, info, x = _gmres(ctx, gpu, A, b, restart=m, rtol=1e-300, max_iter=k, reorth=reorth)
        ref = oracle.gmres(A, b, m=m, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k and info["launches"] == 1
        assert info["outer_iters"] == (k + m - 1) // m
        tol = k * kappa * math.sqrt(n) * U48 * np.max(np.abs(ref["x"]))
        assert np.max(np.abs(x - ref["x"])) <= tol, (G, k)


# ---------------------------------------------------------------------------
# the fused and the general path: the same iteration
# ---------------------------------------------------------------------------
def test_fused_and_general_paths_agree(ctx, gpu):
    n = 640
    A = inputs.spd_matrix(n, 0.01, seed=64)
    b = A @ inputs.solution(n, seed=65)
    kappa, _ = _spd_kappa(A)
    s1, i1, x1 = _cg(ctx, gpu, A, b, rtol=1e-10, fused=1)
    s0, i0, x0 = _cg(ctx, gpu, A, b, rtol=1e-10, fused=0)
    assert s0 == s1 == B.LS_OK
    assert i1["launches"] == 1 and i0["launches"] >= 2 * i0["iters"]
    assert abs(i1["iters"] - i0["iters"]) <= 2
    assert np.linalg.norm(x1 - x0) <= 4 * kappa * 1e-10 * np.linalg.norm(x0)
    A = inputs.nonsym_matrix(n, seed=66)
    b = A @ inputs.solution(n, seed=67)
    s1, i1, x1 = _gmres(ctx, gpu, A, b, rtol=1e-10, restart=10, fused=1)
    s0, i0, x0 = _gmres(ctx, gpu, A, b, rtol=1e-10, restart=10, fused=0)
    assert s0 == s1 == B.LS_OK
    assert abs(i1["iters"] - i0["iters"]) <= 1 and abs(i1["outer_iters"] - i0["outer_iters"]) <= 1
    assert i1["launches"] == 1 < i0["launches"]
    kappa, _ = _svd_kappa(A)
    assert np.linalg.norm(x1 - x0) <= 4 * kappa * 1e-10 * np.linalg.norm(x0)


def test_large_n_takes_the_general_path(ctx, gpu, oracle):
    n = 3000
    A = inputs.spd_matrix(n, 0.1, seed=68)
    b = A @ inputs.solution(n, seed=69)
    st, info, x = _cg(ctx, gpu, A, b, rtol=1e-10)
    assert st == B.LS_OK and info["launches"] >= 2 * info["iters"]
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)


def test_fused_deterministic(ctx, gpu):
    n = 1500
    A = inputs.spd_matrix(n, 0.01, seed=70)
    b = A @ inputs.solution(n, seed=71)
    _, i1, x1 = _cg(ctx, gpu, A, b)
    _, i2, x2 = _cg(ctx, gpu, A, b)
    assert i1["launches"] == 1 and i1["iters"] == i2["iters"] and np.array_equal(x1, x2)


# ---------------------------------------------------------------------------
# edge cases: start values, limits, breakdowns, non-finite input, restarts
# ---------------------------------------------------------------------------
def test_fused_cg_edge_cases(ctx, gpu, oracle):
    n = 203
    A = inputs.spd_matrix(n, 0.1, seed=72)
    xs = inputs.solution(n, seed=72)
    # x0 given: residual start, fewer iterations
    x0 = xs + 1e-6 * inputs.solution(n, seed=73)
    st, warm, x = _cg(ctx, gpu, A, A @ xs, x0=x0)
    _, cold, _ = _cg(ctx, gpu, A, A @ xs)
    assert st == B.LS_OK and warm["iters"] < cold["iters"] and warm["launches"] == 1
    assert np.linalg.norm(oracle.residual(A, A @ xs, x)) <= 1e-10 * np.linalg.norm(A @ xs)
    # exact start: no iteration
    st, info, x = _cg(ctx, gpu, np.eye(n) * 2.0, 2.0 * xs, x0=xs)
    assert st == B.LS_OK and info["iters"] == 0 and np.array_equal(x, xs)
    # b = 0 with a start value: x = 0
    st, info, x = _cg(ctx, gpu, A, np.zeros(n), x0=xs)
    assert st == B.LS_OK and not x.any() and info["iters"] == 0
    # iteration limit
    st, info, x = _cg(ctx, gpu, A, A @ xs, rtol=1e-14, max_iter=3)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 3
    # not SPD: breakdown on the first curvature
    st, info, x = _cg(ctx, gpu, -A, A @ xs)
    assert st == B.LS_BREAKDOWN and info["iters"] == 0
    # non-finite input
    b = A @ xs
    b[7] = np.nan
    assert _cg(ctx, gpu, A, b)[0] == B.LS_ERR_NAN
    # the context is healthy afterwards
    assert _cg(ctx, gpu, A, A @ xs)[0] == B.LS_OK


def test_fused_cg_tight_tolerance(ctx, gpu, oracle):
    """rtol 1e-12 on a cond ~ 4e3 system: the recursive residual runs ahead of
    the true one near the attainable accuracy; the true-residual check keeps
    the solve going (restarting from the true residual) until the true
    residual itself passes."""
    n = 400
    A = inputs.spd_matrix(n, 1e-3, seed=74)
    xs = inputs.solution(n, seed=74)
    b = A @ xs
    st, info, x = _cg(ctx, gpu, A, b, rtol=1e-12, max_iter=20000)
    assert st == B.LS_OK and info["outer_iters"] >= 1 and info["launches"] == 1
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-12 * np.linalg.norm(b)
    ref = oracle.cg(A, b, rtol=1e-12, max_iter=20000)
    _, inv = _spd_kappa(A)
    _converged_ok(oracle, A, b, x, ref["x"], inv, 1e-12)


def test_fused_gmres_edge_cases(ctx, gpu, oracle):
    n = 64
    xs = inputs.solution(n, seed=75)
    st, info, x = _gmres(ctx, gpu, 2.0 * np.eye(n), 2.0 * xs, restart=10)
    assert st == B.LS_OK and info["iters"] == 1 and info["launches"] == 1
    assert np.allclose(x, xs, rtol=0, atol=1e-15)
    A = inputs.nonsym_matrix(n, seed=75)
    st, info, x = _gmres(ctx, gpu, A, np.zeros(n), x0=xs)
    assert st == B.LS_OK and not x.any()
    st, info, x = _gmres(ctx, gpu, A, A @ xs, x0=xs + 1e-9)
    assert st == B.LS_OK and info["iters"] <= 3
    b = A @ xs
    b[0] = np.inf
    assert _gmres(ctx, gpu, A, b)[0] == B.LS_ERR_NAN
    # singular with b outside the range: no false success
    S = np.diag(np.r_[0.0, np.ones(n - 1)])
    st, info, x = _gmres(ctx, gpu, S, np.ones(n), restart=4, max_iter=40)
    assert st in (B.LS_BREAKDOWN, B.LS_NOT_CONVERGED)
    # the largest restart length
    A = inputs.restart_matrix(300, seed=76)
    b = A @ inputs.solution(300, seed=76)
    st, info, x = _gmres(ctx, gpu, A, b, restart=B.LS_MAX_RESTART, rtol=1e-10)
    ref = oracle.gmres(A, b, m=B.LS_MAX_RESTART, rtol=1e-10)
    assert st == B.LS_OK and info["launches"] == 1 and abs(info["iters"] - ref["iters"]) <= 1


def test_fused_in_user_workspace(ctx, gpu, oracle):
    """ls_workspace_size covers the fused layout: a caller buffer of exactly
    that size runs the solve."""
    n = 777
    A = inputs.spd_matrix(n, 0.1, seed=77)
    b = A @ inputs.solution(n, seed=77)
    for method, fn in ((B.LS_METHOD_CG, _cg), (B.LS_METHOD_GMRES, _gmres)):
        nbytes = B.ls_workspace_size(ctx, method, n, 1, B.make_opts(), a_on_device=True)
        buf = torch.empty(nbytes, dtype=torch.uint8, device=gpu)
        assert B.ls_set_workspace(ctx, buf, nbytes) == B.LS_OK
        try:
            st, info, x = fn(ctx, gpu, torch.from_numpy(A).to(gpu), b, rtol=1e-10)
        finally:
            B.ls_set_workspace(ctx, None, 0)
        assert st == B.LS_OK and info["launches"] == 1
        assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
