"""Pins for the oracle's Gaussian elimination and low-precision roundings.

GE is checked against LAPACK (numpy.linalg.solve) and on cases that force
pivoting.  The BF16 and FP8-e4m3 roundings are checked (a) against torch's
own conversions on inputs exactly representable in FP32 (so no double
rounding is involved), (b) by brute force: the result is a representable
value, no representable neighbour is closer, and exact ties go to the even
code, and (c) by round-tripping every FP8 code.
"""
import math

import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import inputs


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_ge_matches_lapack(oracle, n):
    A = inputs.nonsym_matrix(n, seed=n)
    b = A @ inputs.solution(n, seed=n)
    x, st = oracle.ge_solve(A, b)
    assert st == oracle.OK
    x_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


def test_ge_pivoting_and_singular(oracle):
    # zero leading pivot: only solvable with a row exchange
    A = np.array([[0.0, 1.0, 2.0], [1.0, 0.0, 3.0], [4.0, -3.0, 8.0]])
    b = np.array([1.0, 2.0, 3.0])
    x, st = oracle.ge_solve(A, b)
    assert st == oracle.OK
    assert np.allclose(A @ x, b, rtol=0, atol=1e-14)
    # tiny pivot: partial pivoting keeps the solve accurate
    A = np.array([[1e-20, 1.0], [1.0, 1.0]])
    x, st = oracle.ge_solve(A, np.array([1.0, 2.0]))
    assert st == oracle.OK
    assert np.allclose(x, [1.0, 1.0], rtol=1e-15)
    # singular
    x, st = oracle.ge_solve(np.ones((4, 4)), np.ones(4))
    assert st == oracle.BREAKDOWN


# ---------------------------------------------------------------- BF16

def _bf16_neighbours(v):
    """Adjacent BF16 values around a finite BF16 value v (as doubles)."""
    f = np.array([v], dtype=np.float32).view(np.uint32)[0]
    out = []
    for step in (-1, 1):
        u = np.uint32((int(f) >> 16) + step) << np.uint32(16)
        out.append(float(np.array([u], dtype=np.uint32).view(np.float32)[0]))
    return out


def test_bf16_matches_torch_on_fp32_values(oracle):
    r = np.random.default_rng(0)
    x = np.concatenate([r.standard_normal(2000), r.standard_normal(500) * 1e30,
                        r.standard_normal(500) * 1e-30]).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16_round(v) for v in x])
    assert np.array_equal(got, ref)


def test_bf16_nearest_and_ties_to_even(oracle):
    r = np.random.default_rng(1)
    for d in r.standard_normal(3000) * np.exp(r.uniform(-40, 40, 3000)):
        q = oracle.bf16_round(d)
        assert float(np.float32(q)) == q
        assert np.array([q], dtype=np.float32).view(np.uint32)[0] & 0xFFFF == 0
        for nb in _bf16_neighbours(q):
            assert abs(d - q) <= abs(d - nb)
    # exact midpoints between adjacent BF16 values round to the even code
    for v in [1.0, 1.0078125, 3.5, 1e-3, -7.25e10]:
        q = oracle.bf16_round(v)
        lo, hi = _bf16_neighbours(q)
        for other in (lo, hi):
            mid = (q + other) / 2.0
            got = oracle.bf16_round(mid)
            code = int(np.array([got], dtype=np.float32).view(np.uint32)[0]) >> 16
            assert code % 2 == 0 and got in (q, other)
    assert oracle.bf16_round(3.5e38) == math.inf
    assert oracle.bf16_round(-0.0) == 0.0 and math.copysign(1, oracle.bf16_round(-0.0)) < 0


def test_bf16_quant_codes(oracle):
    A = inputs.spd_matrix(16, 0.1, seed=3)
    Q = oracle.quant_bf16(A)
    vals = oracle.decode_bf16(Q).astype(np.float64)
    expect = np.vectorize(oracle.bf16_round)(A)
    assert np.array_equal(vals, expect)
    assert np.all(np.abs(vals - A) <= np.abs(A) * 2.0 ** -8)


# ---------------------------------------------------------------- FP8 e4m3

def test_e4m3_round_trip_all_codes(oracle):
    for c in range(256):
        v = oracle.e4m3_decode(c)
        if math.isnan(v):
            assert c in (0x7F, 0xFF)
            continue
        assert oracle.e4m3_round(v) == v
    assert oracle.e4m3_decode(0x7E) == 448.0
    assert oracle.e4m3_decode(0x01) == 2.0 ** -9
    assert oracle.e4m3_decode(0x08) == 2.0 ** -6


def test_e4m3_matches_torch_in_range(oracle):
    r = np.random.default_rng(2)
    x = np.concatenate([r.uniform(-448, 448, 3000), r.standard_normal(2000),
                        r.standard_normal(1000) * 1e-2]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([oracle.e4m3_round(float(v)) for v in x])
    assert np.array_equal(got, ref)


def test_e4m3_nearest_saturating(oracle):
    finite = sorted({oracle.e4m3_decode(c) for c in range(256)} - {math.nan}
                    - {v for v in [oracle.e4m3_decode(0x7F)]})
    finite = np.array([v for v in finite if not math.isnan(v)])
    r = np.random.default_rng(3)
    for d in r.uniform(-500, 500, 2000):
        q = oracle.e4m3_round(d)
        if abs(d) >= 448.0:
            assert q == math.copysign(448.0, d)
            continue
        best = np.min(np.abs(finite - d))
        assert abs(q - d) == best
    assert oracle.e4m3_round(1e9) == 448.0 and oracle.e4m3_round(-1e9) == -448.0
    assert oracle.e4m3_round(464.0) == 448.0          # beyond the largest finite value
    assert oracle.e4m3_round(1.0625) == 1.0           # tie between 1 and 1.125 -> even
    assert oracle.e4m3_round(1.1875) == 1.25          # tie between 1.125 and 1.25 -> even


def test_fp8_quant_row_scales(oracle):
    A = inputs.nonsym_matrix(24, seed=5)
    Q, s = oracle.quant_fp8(A)
    mx = np.abs(A).max(axis=1)
    assert np.array_equal(s, (mx / 448.0).astype(np.float32))
    dec = oracle.decode_fp8(Q).astype(np.float64) * s[:, None].astype(np.float64)
    # relative error of a 4-significant-bit rounding (normal range)
    big = np.abs(A) >= 2.0 ** -6 * s[:, None]
    assert np.all(np.abs(dec - A)[big] <= np.abs(A)[big] * 2.0 ** -4 * 1.0001)
    # row maxima land on the top of the range
    assert np.all(np.abs(oracle.decode_fp8(Q)).max(axis=1) == 448.0)


@pytest.mark.parametrize("n", [1, 5, 60])
def test_ge_factor_is_partial_pivoting_lu(oracle, n):
    # the exported factors: P A = L U (numpy, FP64) to rounding, |L| <= 1 (the
    # defining property of partial pivoting), y = L^-1 P b, and the solve path
    # (or_ge_solve) gives the back substitution of the same factors
    A = inputs.nonsym_matrix(n, seed=200 + n)
    b = A @ inputs.solution(n, seed=201 + n)
    LU, ipiv, y, st = oracle.ge_factor(A, b)
    assert st == oracle.OK
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA, Pb = A.copy(), b.copy()
    for k in range(n):
        PA[[k, ipiv[k]]] = PA[[ipiv[k], k]]
        Pb[[k, ipiv[k]]] = Pb[[ipiv[k], k]]
        assert ipiv[k] >= k
    assert np.max(np.abs(PA - L @ U)) <= 4 * n * 2.0 ** -52 * np.max(np.abs(A)) * max(1, n)
    assert np.max(np.abs(L)) <= 1.0
    assert np.allclose(L @ y, Pb, rtol=0, atol=1e-12 * np.abs(b).max())
    x, st2 = oracle.ge_solve(A, b)
    assert st2 == oracle.OK
    assert np.allclose(U @ x, y, rtol=0, atol=1e-12 * np.abs(y).max())
