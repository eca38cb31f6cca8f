"""The device path against the hand-derived worked examples of tests/golden:
the same small systems the oracle is pinned to, solved through the C ABI.
The LU factors, pivots and forward-substituted right-hand side are dyadic
and the device elimination is the plain elimination bit for bit, so they
must match exactly; the iterative methods must reach the exact solutions
the derivations give."""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from test_oracle_golden import load

pytestmark = pytest.mark.gpu


def _dev(gpu, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(gpu)


def _solve(fn, ctx, gpu, A, b, **kw):
    x = torch.zeros(len(b), dtype=torch.float64, device=gpu)
    st, info = fn(ctx, _dev(gpu, A), _dev(gpu, b), x, B.make_opts(**kw))
    return st, x.cpu().numpy()


def _close(x, ref, tol=1e-13):
    return np.max(np.abs(x - ref)) <= tol * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prefix", ["", "tie_"])
def test_lu_worked_example_device(ctx, gpu, prefix):
    g = load("lu_3x3.txt")
    A, b = g[prefix + "A"], g[prefix + "b"]
    n = A.shape[0]
    LU = torch.zeros((n, n), dtype=torch.float64, device=gpu)
    ipiv = torch.zeros(n, dtype=torch.int32, device=gpu)
    y = torch.zeros(n, dtype=torch.float64, device=gpu)
    assert B.ls_lu_factor(ctx, _dev(gpu, A), _dev(gpu, b), LU, ipiv, y) == B.LS_OK
    assert np.array_equal(LU.cpu().numpy(), g[prefix + "LU"])
    assert ipiv.cpu().numpy().tolist() == g[prefix + "ipiv"].astype(int).tolist()
    assert np.array_equal(y.cpu().numpy(), g[prefix + "y"])
    st, x = _solve(B.ls_lu_solve, ctx, gpu, A, b)
    assert st == B.LS_OK and _close(x, g[prefix + "x"], 1e-15)


def test_krylov_worked_examples_device(ctx, gpu):
    g = load("cg_2x2.txt")
    st, x = _solve(B.ls_cg_solve, ctx, gpu, g["A"], g["b"], rtol=1e-12)
    assert st == B.LS_OK and _close(x, g["x2"])
    g = load("gmres_2x2.txt")
    st, x = _solve(B.ls_gmres_solve, ctx, gpu, g["A"], g["b"], rtol=1e-12, restart=30)
    assert st == B.LS_OK and _close(x, g["x2"])
    g = load("bicgstab_diag2.txt")
    st, x = _solve(B.ls_bicgstab_solve, ctx, gpu, g["A"], g["b"], rtol=1e-12)
    assert st == B.LS_OK and _close(x, np.linalg.solve(g["A"], g["b"]))     # [1/2, 1/4]


def test_stationary_worked_examples_device(ctx, gpu):
    g = load("jacobi_gs_2x2.txt")
    for fn in (B.ls_jacobi_solve, B.ls_gauss_seidel_solve):
        st, x = _solve(fn, ctx, gpu, g["A"], g["b"], rtol=1e-12)
        assert st == B.LS_OK and _close(x, np.ones(2), 1e-11)
