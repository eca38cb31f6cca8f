"""The device LU runs the right-looking elimination by panels (the panel's
pivot steps on its own columns, its row swaps on the other columns, the
pivot rows right of the panel, then the trailing block).  The claim that
makes its factors equal to the plain elimination bit for bit is that this
only regroups the operations: every element still receives
a_ij - l_it u_tj for t = 0, 1, ... in order, each product and difference
rounded once.  This CPU test replays that schedule in numpy (products and
differences as separate FP64 operations) for several panel widths and
ragged sizes, and compares it with the oracle's plain elimination exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1511_07207_gb300 import inputs


def blocked_elimination(A, b, nb):
    """[A | b] eliminated panel by panel; returns (LU, ipiv, y)."""
    n = A.shape[0]
    W = np.concatenate([A, b[:, None]], axis=1).astype(np.float64)
    ipiv = np.zeros(n, dtype=np.int64)
    for k0 in range(0, n, nb):
        k1 = min(n, k0 + nb)
        # the panel's steps on its own columns
        for k in range(k0, k1):
            v = k + int(np.argmax(np.abs(W[k:, k])))   # the first row of the largest |a_ik|
            ipiv[k] = v
            W[[k, v], k0:k1] = W[[v, k], k0:k1]
            piv = W[k, k]
            assert piv != 0.0
            l = W[k + 1:, k] / piv
            W[k + 1:, k] = l
            W[k + 1:, k + 1:k1] = W[k + 1:, k + 1:k1] - np.outer(l, W[k, k + 1:k1])
        # the panel's swaps on the other columns, in step order
        other = np.r_[0:k0, k1:n + 1]
        for t in range(k0, k1):
            v = ipiv[t]
            rows = W[[t, v]][:, other]
            W[t, other], W[v, other] = rows[1], rows[0]
        # the pivot rows right of the panel: u_rj -= l_rt u_tj, t in order
        for r in range(k0 + 1, k1):
            for t in range(k0, r):
                W[r, k1:] = W[r, k1:] - W[r, t] * W[t, k1:]
        # the trailing block: the panel's updates in step order
        for t in range(k0, k1):
            W[k1:, k1:] = W[k1:, k1:] - np.outer(W[k1:, t], W[t, k1:])
    return W[:, :n], ipiv, W[:, n]


@pytest.mark.parametrize("n,nb", [(1, 32), (5, 2), (33, 32), (70, 32), (100, 8), (129, 32)])
def test_blocked_schedule_equals_plain_elimination(n, nb):
    A = inputs.nonsym_matrix(n, seed=300 + n)
    b = A @ inputs.solution(n, seed=300 + n)
    LU, ipiv, y = blocked_elimination(A, b, nb)
    LU0, ipiv0, y0, st = oracle.default().ge_factor(A, b)
    assert st == 0
    assert ipiv.tolist() == ipiv0.tolist()
    assert np.array_equal(LU, LU0)          # bit for bit
    assert np.array_equal(y, y0)


def test_blocked_schedule_with_ties_equals_plain_elimination():
    rng = np.random.default_rng(7)
    n = 48
    A = rng.integers(-3, 4, size=(n, n)).astype(np.float64) + 8 * np.eye(n) * rng.integers(0, 2, n)
    A[np.diag_indices(n)] += (A.diagonal() == 0)          # nonsingular enough for the test
    b = A @ np.ones(n)
    LU0, ipiv0, y0, st = oracle.default().ge_factor(A, b)
    if st != 0:
        pytest.skip("singular draw")
    LU, ipiv, y = blocked_elimination(A, b, 16)
    assert ipiv.tolist() == ipiv0.tolist()
    assert np.array_equal(LU, LU0) and np.array_equal(y, y0)
