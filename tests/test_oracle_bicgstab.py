"""Pins for the oracle's BiCGSTAB (CPU only).

Independent checks: LAPACK solves of nonsymmetric and SPD systems; the two
orthogonality relations that define the step lengths in exact arithmetic
(alpha makes s = r - alpha v orthogonal to the shadow residual r^, and omega
minimises ||s - omega t||, so the new residual is orthogonal to t); one
product for a multiple of the identity; the step lengths alpha_k of plain BiCG
(Fletcher's form, run here in numpy with A^T and the same shadow residual),
which BiCGSTAB reproduces in exact arithmetic; a breakdown that the mathematics
forces (r^.v = 0 at the first step); the iteration limit; and a convergence
rate no worse than that of GMRES on the same well-conditioned matrix (two
products per BiCGSTAB step, each reducing the residual at least as fast as
one GMRES step does on a spectrum in a disk of radius 1/2 around 2).
"""
import numpy as np
import pytest

from paper_1511_07207_gb300 import inputs


def _cond(A):
    s = np.linalg.svd(A, compute_uv=False)
    return s[0] / s[-1]


@pytest.mark.parametrize("n", [1, 2, 17, 64, 200])
def test_bicgstab_matches_lapack(oracle, n):
    A = inputs.nonsym_matrix(n, seed=300 + n)
    xs = inputs.solution(n, seed=300 + n)
    b = A @ xs
    out = oracle.bicgstab(A, b, rtol=1e-12)
    assert out["status"] == oracle.OK
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(out["x"] - ref) <= 4 * _cond(A) * 1e-12 * np.linalg.norm(ref)
    assert out["rel_res"] <= 1e-12


def test_bicgstab_spd(oracle):
    n = 120
    A = inputs.spd_matrix(n, 0.1, seed=3)
    b = A @ inputs.solution(n, seed=3)
    out = oracle.bicgstab(A, b, rtol=1e-11)
    assert out["status"] == oracle.OK
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(out["x"] - ref) <= 4 * _cond(A) * 1e-11 * np.linalg.norm(ref)


def test_bicgstab_step_orthogonality(oracle):
    n = 150
    A = inputs.nonsym_matrix(n, seed=8)
    b = A @ inputs.solution(n, seed=8)
    out = oracle.bicgstab(A, b, rtol=1e-12, trace=True)
    assert out["status"] == oracle.OK and len(out["shs"]) >= 5
    assert np.max(np.abs(out["shs"])) <= 1e-9      # r^ . s = 0
    assert np.max(np.abs(out["rt"])) <= 1e-9       # r_new . t = 0


def _bicg_alphas(A, b, steps):
    """Plain BiCG with the transpose (an independent algorithm): its alphas."""
    x = np.zeros_like(b)
    r = b - A @ x
    rs = r.copy()
    p, ps = r.copy(), rs.copy()
    out = []
    for _ in range(steps):
        Ap = A @ p
        a = (rs @ r) / (ps @ Ap)
        out.append(a)
        r_new = r - a * Ap
        rs_new = rs - a * (A.T @ ps)
        beta = (rs_new @ r_new) / (rs @ r)
        r, rs = r_new, rs_new
        p = r + beta * p
        ps = rs + beta * ps
    return np.array(out)


def test_bicgstab_alphas_equal_bicg(oracle):
    n = 80
    A = inputs.nonsym_matrix(n, seed=12)
    b = A @ inputs.solution(n, seed=12)
    out = oracle.bicgstab(A, b, rtol=1e-12, trace=True)
    k = min(6, len(out["alphas"]))
    ref = _bicg_alphas(A, b, k)
    assert np.allclose(out["alphas"][:k], ref, rtol=1e-7, atol=0)


def test_bicgstab_identity_multiple_one_product(oracle):
    n = 9
    A = 3.0 * np.eye(n)
    b = np.arange(1.0, n + 1)
    out = oracle.bicgstab(A, b, rtol=1e-12)
    assert out["status"] == oracle.OK and out["iters"] == 1
    assert np.allclose(out["x"], b / 3.0, rtol=0, atol=1e-15)


def test_bicgstab_breakdown_and_limits(oracle):
    A = np.array([[0.0, 1.0], [-1.0, 0.0]])          # rotation: r^.A r^ = 0
    out = oracle.bicgstab(A, np.array([1.0, 0.0]), rtol=1e-12)
    assert out["status"] == oracle.BREAKDOWN
    n = 50
    A = inputs.nonsym_matrix(n, seed=1)
    b = A @ inputs.solution(n, seed=1)
    out = oracle.bicgstab(A, b, rtol=1e-14, max_iter=3)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters"] == 3
    out = oracle.bicgstab(A, np.zeros(n))
    assert out["status"] == oracle.OK and out["iters"] == 0 and not out["x"].any()


def test_bicgstab_rate_against_gmres(oracle):
    n = 300
    A = inputs.nonsym_matrix(n, seed=44)
    b = A @ inputs.solution(n, seed=44)
    bi = oracle.bicgstab(A, b, rtol=1e-10)
    gm = oracle.gmres(A, b, m=60, rtol=1e-10)
    assert bi["status"] == gm["status"] == oracle.OK
    assert bi["iters"] <= 2 * gm["iters"] + 4
