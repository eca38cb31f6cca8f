"""GPU parity of the mixed-precision CG (BF16 / FP8-e4m3 / FP32 storage of A,
FP32 inner CG, FP64 outer flexible CG or classic refinement) with the oracle.

The FP64 outer loop is driven by the FP64 residual, so the result must meet
the same FP64 tolerance as the plain solver: true relative residual (computed
by the oracle) <= rtol, error against the oracle's FP64 solution within
kappa * rtol.  Outer step counts must match the oracle's mixed solver to
within a few steps (the inner FP32 iterates differ by rounding order).
Storage that cannot represent A well enough (FP8 at cond ~ 4e3) must report
a failure status, never a false success.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu

PREC = {"bf16": B.LS_BF16_IR, "fp8": B.LS_FP8_IR, "f32": B.LS_F32_IR}
MODE = {"fcg": B.LS_REFINE_FCG, "ir": B.LS_REFINE_IR}


def _solve(ctx, gpu, A, b, precision, mode, x0=None, **kw):
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(gpu)
    bd = torch.from_numpy(b).to(gpu)
    xd = torch.from_numpy(x0.copy() if x0 is not None else np.zeros(len(b))).to(gpu)
    o = B.make_opts(precision=PREC[precision], refine=MODE[mode], x0_given=int(x0 is not None),
                    **kw)
    st, info = B.ls_cg_solve(ctx, Ad, bd, xd, o)
    return st, info, xd.cpu().numpy()


def _stored(oracle, A, precision):
    if precision == "bf16":
        return oracle.decode_bf16(oracle.quant_bf16(A)), None
    if precision == "fp8":
        Q, s = oracle.quant_fp8(A)
        return oracle.decode_fp8(Q), s
    return A.astype(np.float32), None


@pytest.mark.parametrize("precision", ["bf16", "fp8", "f32"])
@pytest.mark.parametrize("mode", ["fcg", "ir"])
@pytest.mark.parametrize("n", [257, 1000])
def test_mixed_well_conditioned(ctx, gpu, oracle, precision, mode, n):
    A = inputs.spd_matrix(n, 0.1, seed=n + 1)          # cond ~ 40
    xs = inputs.solution(n, seed=n + 1)
    b = A @ xs
    extra = {"inner_rtol": 1e-2} if mode == "ir" else {}
    st, info, x = _solve(ctx, gpu, A, b, precision, mode, rtol=1e-10, **extra)
    assert st == B.LS_OK, B.ls_strerror(st)
    nb = np.linalg.norm(b)
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * nb
    ref = oracle.cg(A, b, rtol=1e-12)
    ev = np.linalg.eigvalsh(A)
    kap = ev[-1] / ev[0]
    assert np.linalg.norm(x - ref["x"]) <= 4 * kap * 1e-10 * np.linalg.norm(ref["x"])
    Af, s = _stored(oracle, A, precision)
    om = oracle.mixed_cg(A, Af, b, scale=s, rtol=1e-10, inner_iters=25, mode=mode, **extra)
    assert om["status"] == oracle.OK
    assert abs(info["outer_iters"] - om["outer"]) <= 3
    assert info["iters"] <= 25 * info["outer_iters"]


def test_fcg_bf16_ill_conditioned(ctx, gpu, oracle):
    n = 1024
    A = inputs.spd_matrix(n, 1e-3, seed=3)             # cond ~ 4e3
    xs = inputs.solution(n, seed=3)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, b, "bf16", "fcg", rtol=1e-10)
    assert st == B.LS_OK
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    Af, _ = _stored(oracle, A, "bf16")
    om = oracle.mixed_cg(A, Af, b, rtol=1e-10, inner_iters=25, mode="fcg")
    assert om["status"] == oracle.OK
    assert abs(info["outer_iters"] - om["outer"]) <= 3
    plain = oracle.cg(A, b, rtol=1e-10)
    assert info["outer_iters"] < plain["iters"] / 4   # far fewer FP64 passes over A


def test_fp8_ill_conditioned_never_false_success(ctx, gpu, oracle):
    n = 1024
    A = inputs.spd_matrix(n, 1e-3, seed=3)
    b = A @ inputs.solution(n, seed=3)
    for mode in ("fcg", "ir"):
        st, info, x = _solve(ctx, gpu, A, b, "fp8", mode, rtol=1e-10, max_iter=40)
        rel = np.linalg.norm(oracle.residual(A, b, x)) / np.linalg.norm(b)
        if st == B.LS_OK:
            assert rel <= 1e-10
        else:
            assert st in (B.LS_NOT_CONVERGED, B.LS_BREAKDOWN)


def test_mixed_edge_cases(ctx, gpu, oracle):
    n = 300
    A = inputs.spd_matrix(n, 0.1, seed=4)
    xs = inputs.solution(n, seed=4)
    b = A @ xs
    st, info, x = _solve(ctx, gpu, A, np.zeros(n), "bf16", "fcg", x0=xs)
    assert st == B.LS_OK and not x.any()
    st, info, x = _solve(ctx, gpu, A, b, "bf16", "fcg", x0=xs.copy())
    assert st == B.LS_OK and info["outer_iters"] == 0
    st, info, x = _solve(ctx, gpu, A, b, "bf16", "fcg", x0=xs + 1e-3)
    assert st == B.LS_OK
    assert np.linalg.norm(oracle.residual(A, b, x)) <= 1e-10 * np.linalg.norm(b)
    bn = b.copy()
    bn[3] = np.nan
    st, info, x = _solve(ctx, gpu, A, bn, "bf16", "fcg")
    assert st == B.LS_ERR_NAN
    st, info, x = _solve(ctx, gpu, A, b, "bf16", "fcg", rtol=1e-14, max_iter=2)
    assert st == B.LS_NOT_CONVERGED and info["outer_iters"] == 2
    st, info, x = _solve(ctx, gpu, A, b, "bf16", "fcg", inner_iters=0)
    assert st in (B.LS_OK, B.LS_NOT_CONVERGED, B.LS_BREAKDOWN)
    st, info, x = _solve(ctx, gpu, A, b, "bf16", "fcg")
    assert st == B.LS_OK
    # GMRES has no mixed path
    Ad = torch.from_numpy(A).to(gpu)
    xd = torch.zeros(n, dtype=torch.float64, device=gpu)
    st, _ = B.ls_gmres_solve(ctx, Ad, torch.from_numpy(b).to(gpu), xd,
                             B.make_opts(precision=B.LS_BF16_IR))
    assert st == B.LS_ERR_UNSUPPORTED
