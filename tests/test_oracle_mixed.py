"""Pins for the oracle's mixed-precision path (CPU only).

The FP32 inner CG is checked against a LAPACK solve of the same stored
matrix; the FP64 outer loop (flexible CG, or classic refinement) is checked
by the FP64 true residual computed here with numpy and by the error against
a LAPACK solve of the FP64 system.  Flexible CG must keep its stored
directions mutually A-conjugate, which is checked directly.
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _stored(oracle, A, precision):
    if precision == "bf16":
        return oracle.decode_bf16(oracle.quant_bf16(A)), None
    Q, s = oracle.quant_fp8(A)
    return oracle.decode_fp8(Q), s


def test_inner_cg_f32_solves_stored_matrix(oracle):
    n = 96
    A = inputs.spd_matrix(n, 0.1, seed=8)
    Af, _ = _stored(oracle, A, "bf16")
    rhs = inputs.solution(n, seed=8).astype(np.float32)
    z, k = oracle.cg_f32(Af, rhs, iters=200, inner_rtol=1e-6)
    ref = np.linalg.solve(Af.astype(np.float64), rhs.astype(np.float64))
    assert k < 200
    assert np.linalg.norm(z - ref) <= 1e-4 * np.linalg.norm(ref)
    # a fixed count runs exactly that many iterations
    z, k = oracle.cg_f32(Af, rhs, iters=7)
    assert k == 7
    # with an FP8 row scale the inner operator is diag(s) Q
    Aq, s = _stored(oracle, A, "fp8")
    z, k = oracle.cg_f32(Aq, rhs, iters=400, inner_rtol=1e-6, scale=s)
    M = s[:, None].astype(np.float64) * Aq.astype(np.float64)
    ref = np.linalg.solve(M, rhs.astype(np.float64))
    assert np.linalg.norm(z - ref) <= 1e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision,mode", [("bf16", "fcg"), ("bf16", "ir"),
                                            ("fp8", "fcg"), ("fp8", "ir")])
def test_mixed_well_conditioned(oracle, precision, mode):
    n = 256
    A = inputs.spd_matrix(n, 0.1, seed=12)          # cond ~ 40
    xs = inputs.solution(n, seed=12)
    b = A @ xs
    Af, s = _stored(oracle, A, precision)
    out = oracle.mixed_cg(A, Af, b, scale=s, rtol=1e-10, inner_iters=25,
                          mode=mode, inner_rtol=1e-2 if mode == "ir" else 0.0)
    assert out["status"] == oracle.OK
    rel = np.linalg.norm(b - A @ out["x"]) / np.linalg.norm(b)
    assert rel <= 1e-10
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(out["x"] - x_ref) <= 100 * 1e-10 * np.linalg.norm(x_ref)
    assert out["outer"] <= 20


def test_fcg_ill_conditioned_bf16(oracle):
    n = 384
    A = inputs.spd_matrix(n, 1e-3, seed=14)         # cond ~ 4e3
    b = A @ inputs.solution(n, seed=14)
    Af, _ = _stored(oracle, A, "bf16")
    out = oracle.mixed_cg(A, Af, b, rtol=1e-10, inner_iters=25, mode="fcg",
                          directions=True)
    assert out["status"] == oracle.OK
    # flexible CG keeps its FP64 directions A-conjugate (full orthogonalisation)
    P = out["P"][: out["outer"]]
    AP = P @ A
    D = np.sqrt(np.einsum("ij,ij->i", P, AP))
    C = np.abs(P @ AP.T) / np.outer(D, D)
    np.fill_diagonal(C, 0.0)
    assert C.max() <= 1e-6
    assert np.linalg.norm(b - A @ out["x"]) <= 1e-10 * np.linalg.norm(b)
    # fewer FP64 matrix passes than plain FP64 CG needs
    plain = oracle.cg(A, b, rtol=1e-10)
    assert out["outer"] < plain["iters"] / 4


def test_classic_ir_never_claims_false_convergence(oracle):
    n = 384
    A = inputs.spd_matrix(n, 1e-3, seed=14)
    b = A @ inputs.solution(n, seed=14)
    Aq, s = _stored(oracle, A, "fp8")
    out = oracle.mixed_cg(A, Aq, b, scale=s, rtol=1e-10, inner_iters=25,
                          mode="ir", inner_rtol=1e-2, max_outer=30)
    rel = np.linalg.norm(b - A @ out["x"]) / np.linalg.norm(b)
    if out["status"] == oracle.OK:
        assert rel <= 1e-10
    else:
        assert out["status"] in (oracle.NOT_CONVERGED, oracle.BREAKDOWN)
