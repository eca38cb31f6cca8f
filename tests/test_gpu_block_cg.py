"""GPU parity of block CG (ls_block_cg_solve) with the oracle.

The iterates are the oracle's up to rounding.  At a fixed step count the
block iterate is the A-norm minimiser over the block Krylov space, which
rounding perturbs only at the level of the products, so the comparison after
k steps is element by element.  To a tolerance: every column's true residual
(computed by the oracle) reaches rtol and the step counts agree within a few.
Edge cases: s = 1 (CG), s = 16, n = 1, ragged n, an initial guess, an exact
initial guess, dependent and zero columns (breakdown), the iteration limit,
NaN input, unsupported precision and s, both product modes, host buffers.
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
        Bd = torch.from_numpy(np.ascontiguousarray(Bm.T)).to(gpu).t()        # columns contiguous
        Xd = torch.from_numpy(np.ascontiguousarray((X0 if X0 is not None else np.zeros((n, s))).T)).to(gpu).t()
    else:
        Ad, Bd = np.ascontiguousarray(A), np.asfortranarray(Bm)
        Xd = np.asfortranarray(X0.copy() if X0 is not None else np.zeros((n, s)))
    o = B.make_opts(x0_given=int(X0 is not None), **kw)
    st, info = B.ls_block_cg_solve(ctx, Ad, Bd, Xd, o)
    X = Xd.cpu().numpy() if on_device else np.array(Xd)
    return st, info, X


def _true_rel(oracle, A, Bm, X):
    return max(np.linalg.norm(oracle.residual(A, Bm[:, j], X[:, j])) / np.linalg.norm(Bm[:, j])
               for j in range(Bm.shape[1]))


def _oracle_for(oracle, deflate):
    return oracle.block_cg_deflated if deflate else oracle.block_cg


@pytest.mark.parametrize("deflate", [0, 1])
@pytest.mark.parametrize("n,s", [(1, 1), (33, 1), (257, 3), (1000, 8), (2049, 16)])
def test_block_cg_matches_oracle(ctx, gpu, oracle, n, s, deflate):
    A = inputs.spd_matrix(n, 0.1, seed=70 + n)
    Bm = A @ inputs.solution(n, seed=71 + n, nrhs=s).reshape(n, s)
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-10, deflate=deflate)
    ref = _oracle_for(oracle, deflate)(A, Bm, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    tr = _true_rel(oracle, A, Bm, X)
    assert tr <= 1e-10
    assert abs(info["rel_res"] - tr) <= 1e-3 * tr + 1e-14
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 20
    assert info["launches"] >= 2 * info["iters"]


@pytest.mark.parametrize("deflate", [0, 1])
@pytest.mark.parametrize("f64_matvec", [0, 1])
@pytest.mark.parametrize("n,s", [(200, 4), (777, 6)])
def test_block_cg_fixed_count_elementwise(ctx, gpu, oracle, n, s, f64_matvec, deflate):
    A = inputs.spd_matrix(n, 0.1, seed=80 + n)
    Bm = A @ inputs.solution(n, seed=81 + n, nrhs=s).reshape(n, s)
    for k in (1, 2, 5):
        st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-300, max_iter=k, f64_matvec=f64_matvec, deflate=deflate)
        ref = _oracle_for(oracle, deflate)(A, Bm, rtol=1e-300, max_iter=k)
        assert st == B.LS_NOT_CONVERGED == ref["status"]
        assert info["iters"] == ref["iters"] == k
        assert np.max(np.abs(X - ref["X"])) <= 1e-11 * np.max(np.abs(ref["X"]))


def test_block_cg_fewer_steps_than_cg_and_host_buffers(ctx, gpu, oracle):
    n, s = 1500, 8
    A = inputs.spd_matrix(n, 1e-3, seed=90)          # cond ~ 4e3
    Bm = A @ inputs.solution(n, seed=91, nrhs=s).reshape(n, s)
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-10)
    assert st == B.LS_OK and _true_rel(oracle, A, Bm, X) <= 1e-10
    cg_iters = oracle.cg(A, Bm[:, 0], rtol=1e-10)["iters"]
    assert info["iters"] < cg_iters
    st2, info2, X2 = _solve(ctx, gpu, A, Bm, on_device=False, rtol=1e-10)
    assert st2 == B.LS_OK and info2["iters"] == info["iters"] and np.array_equal(X, X2)


def test_block_cg_initial_guess(ctx, gpu, oracle):
    n, s = 400, 4
    A = inputs.spd_matrix(n, 0.1, seed=92)
    Xs = inputs.solution(n, seed=93, nrhs=s).reshape(n, s)
    Bm = A @ Xs
    st, cold, _ = _solve(ctx, gpu, A, Bm, rtol=1e-10)
    st, info, X = _solve(ctx, gpu, A, Bm, X0=Xs + 1e-6 * inputs.solution(n, seed=94, nrhs=s).reshape(n, s),
                         rtol=1e-10)
    assert st == B.LS_OK and info["iters"] < cold["iters"] and _true_rel(oracle, A, Bm, X) <= 1e-10
    st, info, X = _solve(ctx, gpu, A, Bm, X0=Xs.copy(), rtol=1e-10)
    assert st == B.LS_OK and info["iters"] == 0


def test_block_cg_edge_cases(ctx, gpu):
    n = 64
    A = inputs.spd_matrix(n, 0.5, seed=95)
    b = A @ inputs.solution(n, seed=95)
    st, info, X = _solve(ctx, gpu, A, np.stack([b, b], 1), deflate=0)      # O'Leary's form
    assert st == B.LS_BREAKDOWN
    st, info, X = _solve(ctx, gpu, A, np.stack([b, np.zeros(n)], 1), deflate=0)
    assert st == B.LS_BREAKDOWN
    st, info, X = _solve(ctx, gpu, A, np.stack([b, b], 1))                 # the deflating form
    assert st == B.LS_OK and np.array_equal(X[:, 0], X[:, 1])
    st, info, X = _solve(ctx, gpu, A, np.stack([b, np.zeros(n)], 1))
    assert st == B.LS_OK and not X[:, 1].any()
    st, info, X = _solve(ctx, gpu, A, np.zeros((n, 3)))
    assert st == B.LS_OK and not X.any() and info["iters"] == 0
    Bm = A @ inputs.solution(n, seed=96, nrhs=3).reshape(n, 3)
    st, info, X = _solve(ctx, gpu, A, Bm, rtol=1e-300, max_iter=2)
    assert st == B.LS_NOT_CONVERGED and info["iters"] == 2
    bad = Bm.copy()
    bad[3, 1] = np.nan
    st, info, X = _solve(ctx, gpu, A, bad)
    assert st == B.LS_ERR_NAN
    st, info, X = _solve(ctx, gpu, A, Bm, precision=B.LS_BF16_IR)
    assert st == B.LS_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        B.ls_block_cg_solve(ctx, A, Bm, Bm.copy())       # not column-major
    big = np.asfortranarray(np.zeros((n, 17)))
    st, _ = B.ls_block_cg_solve(ctx, np.ascontiguousarray(A), big, big.copy(order="F"))
    assert st == B.LS_ERR_ARG


@pytest.mark.parametrize("f64_matvec", [0, 1])
def test_deflation_of_dependent_zero_and_duplicate_columns(ctx, gpu, oracle, f64_matvec):
    """A block whose residual has dependent columns (b0 + 2 b1), a zero column
    and a duplicate: O'Leary's form breaks down, the deflating form drops the
    dependent directions and converges; every column reaches the tolerance,
    agrees with the oracle's deflating block CG within the residual bound,
    and the dependent column's solution is the same combination of the
    others' (to the solve's accuracy)."""
    n = 500
    A = inputs.spd_matrix(n, 0.1, seed=97)
    Bi = A @ inputs.solution(n, seed=98, nrhs=3).reshape(n, 3)
    Bd = np.column_stack([Bi[:, 0], Bi[:, 1], Bi[:, 0] + 2 * Bi[:, 1], np.zeros(n), Bi[:, 2], Bi[:, 1]])
    st0, _, _ = _solve(ctx, gpu, A, Bd, rtol=1e-10, deflate=0, f64_matvec=f64_matvec)
    assert st0 == B.LS_BREAKDOWN
    st, info, X = _solve(ctx, gpu, A, Bd, rtol=1e-10, f64_matvec=f64_matvec)
    ref = oracle.block_cg_deflated(A, Bd, rtol=1e-10)
    assert st == B.LS_OK == ref["status"]
    nz = [0, 1, 2, 4, 5]
    assert _true_rel(oracle, A, Bd[:, nz], X[:, nz]) <= 1e-10
    assert not X[:, 3].any()
    inv = 1.0 / np.linalg.eigvalsh(A)[0]
    for j in nz:
        rg = np.linalg.norm(oracle.residual(A, Bd[:, j], X[:, j]))
        ro = np.linalg.norm(oracle.residual(A, Bd[:, j], ref["X"][:, j]))
        assert np.max(np.abs(X[:, j] - ref["X"][:, j])) <= inv * (rg + ro), j
    sc = np.max(np.abs(X))
    assert np.max(np.abs(X[:, 2] - (X[:, 0] + 2 * X[:, 1]))) <= 1e-8 * sc
    assert abs(info["iters"] - ref["iters"]) <= 2 + ref["iters"] // 20


def test_deflation_when_columns_converge_at_different_times(ctx, gpu, oracle):
    """Columns scaled over ten orders of magnitude and one column already solved
    by the initial guess: the deflating form keeps going on the others and
    every column reaches its own tolerance."""
    n, s = 800, 5
    A = inputs.spd_matrix(n, 0.05, seed=99)
    Xs = inputs.solution(n, seed=100, nrhs=s).reshape(n, s) * np.array([1.0, 1e-5, 1e5, 1.0, 1.0])
    Bm = A @ Xs
    X0 = np.zeros((n, s))
    X0[:, 3] = np.linalg.solve(A, Bm[:, 3])
    st, info, X = _solve(ctx, gpu, A, Bm, X0=X0, rtol=1e-10)
    assert st == B.LS_OK
    assert _true_rel(oracle, A, Bm, X) <= 1e-10

