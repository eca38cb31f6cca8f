"""The oracle against worked examples derived by hand (tests/golden/*.txt).

Each fixture is a small system whose iterates or factors were worked out in
exact rational arithmetic from the method's definition; the derivation and
the passage of the paper it follows are written at the top of the file.
Dyadic values are exact in FP64 and are compared exactly; the others within
a few units of rounding.  The fixtures were written by hand, not by running
either implementation.
"""
import pathlib
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = pathlib.Path(__file__).resolve().parent / "golden"


def load(name):
    """key = numbers: space-separated rationals, matrix rows separated by ';'."""
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, val = (s.strip() for s in line.split("=", 1))
        rows = [[float(Fraction(t)) for t in r.split()] for r in val.split(";")]
        out[key] = np.array(rows[0] if len(rows) == 1 else rows)
    return out


@pytest.fixture(scope="module")
def o():
    return oracle.default()


def close(a, b, ulps=8):
    return np.all(np.abs(np.asarray(a) - np.asarray(b)) <= ulps * np.finfo(float).eps * np.maximum(1.0, np.abs(b)))


def test_fixture_parser():
    g = load("lu_3x3.txt")
    assert g["A"].shape == (3, 3) and g["b"].shape == (3,)
    assert g["LU"][1, 0] == 0.25 and g["tie_ipiv"].tolist() == [0, 1]


def test_cg_worked_example(o):
    g = load("cg_2x2.txt")
    r1 = o.cg(g["A"], g["b"], rtol=1e-30, max_iter=1, history=True)
    assert np.array_equal(r1["x"], g["x1"])                   # dyadic: exact
    assert np.array_equal(r1["R"][1], g["r1"])
    assert np.array_equal(r1["P"][1], g["p1"])
    r2 = o.cg(g["A"], g["b"], rtol=1e-14, max_iter=2)
    assert r2["status"] == 0 and r2["iters"] == 2
    assert close(r2["x"], g["x2"])


def test_gmres_worked_example(o):
    g = load("gmres_2x2.txt")
    r1 = o.gmres(g["A"], g["b"], m=2, rtol=1e-30, max_iter=1)
    assert close(r1["x"], g["x1"])                            # formed through 1/sqrt(2): rounded
    assert close(r1["rel_res"] ** 2, g["res1_sq"])
    assert close(r1["est"] ** 2, g["res1_sq"])                # the Givens estimate is the true residual
    r2 = o.gmres(g["A"], g["b"], m=2, rtol=1e-30, max_iter=2, first_cycle=True)
    assert r2["k"] == 2 and r2["cycles"] == 1
    assert np.array_equal(r2["V"][:, 0], g["v1"]) and np.array_equal(r2["V"][:, 1], g["v2"])
    assert np.array_equal(r2["H"], g["H"])
    assert close(r2["x"], g["x2"])


def test_bicgstab_worked_example(o):
    g = load("bicgstab_diag2.txt")
    half = o.bicgstab(g["A"], g["b"], rtol=1e-30, max_iter=1, trace=True)   # one product
    assert close(half["alphas"][0], g["alpha"])
    assert close(half["x"], g["x_half"])
    full = o.bicgstab(g["A"], g["b"], rtol=1e-30, max_iter=2)               # one full step
    assert close(full["x"], g["x1"])
    assert close(g["b"] - g["A"] @ full["x"], g["r1"])


def test_jacobi_gauss_seidel_worked_example(o):
    g = load("jacobi_gs_2x2.txt")
    # max_iter = k measures the residual of k iterates and returns the last one, x_{k-1}
    assert np.array_equal(o.jacobi(g["A"], g["b"], rtol=1e-30, max_iter=2)["x"], g["jacobi_x1"])
    assert np.array_equal(o.jacobi(g["A"], g["b"], rtol=1e-30, max_iter=3)["x"], g["jacobi_x2"])
    assert np.array_equal(o.gauss_seidel(g["A"], g["b"], rtol=1e-30, max_iter=2)["x"], g["gs_x1"])
    assert np.array_equal(o.gauss_seidel(g["A"], g["b"], rtol=1e-30, max_iter=3)["x"], g["gs_x2"])


@pytest.mark.parametrize("prefix", ["", "tie_"])
def test_lu_worked_example(o, prefix):
    g = load("lu_3x3.txt")
    LU, ipiv, y, st = o.ge_factor(g[prefix + "A"], g[prefix + "b"])
    assert st == 0
    assert np.array_equal(LU, g[prefix + "LU"])               # dyadic: exact
    assert ipiv.tolist() == g[prefix + "ipiv"].astype(int).tolist()
    assert np.array_equal(y, g[prefix + "y"])
    x, st = o.ge_solve(g[prefix + "A"], g[prefix + "b"])
    assert st == 0 and np.array_equal(x, g[prefix + "x"])
