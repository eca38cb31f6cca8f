"""The device Cholesky factorization runs by panels: the panel's steps on its
own columns (l_jk formed by every warp as w_jk / l_kk from the unchanged
column k, the l's collected in a panel buffer), then the trailing lower
triangle, with b^T carried as an extra row so that the last row becomes
y = L^-1 b.  The claim that makes L and y equal to the plain
column-by-column factorization and forward substitution bit for bit is that
this only regroups the operations.  This CPU test replays that schedule in
numpy (products and differences as separate FP64 operations) and compares it
with the oracle exactly."""
import numpy as np
import pytest

import oracle
from paper_1511_07207_gb300 import inputs


def panel_schedule(A, b, nb):
    n = A.shape[0]
    W = np.zeros((n + 1, n))
    W[:n] = np.tril(A)
    W[n] = b
    for k0 in range(0, n, nb):
        k1 = min(n, k0 + nb)
        Lp = np.zeros((n + 1, nb))
        for k in range(k0, k1):                       # the panel's steps
            piv = W[k, k]
            assert piv > 0.0
            lkk = np.sqrt(piv)
            Lp[k, k - k0] = lkk
            ljk = W[k + 1:k1, k] / lkk                # every warp forms these from column k
            for i in range(k + 1, n + 1):
                lik = W[i, k] / lkk
                Lp[i, k - k0] = lik
                jmax = min(k1, i + 1, n)              # panel columns j <= i (and j < n)
                if jmax > k + 1:
                    W[i, k + 1:jmax] = W[i, k + 1:jmax] - lik * ljk[: jmax - k - 1]
        for t in range(k1 - k0):                      # the trailing lower triangle, steps in order
            W[k1:n + 1, k1:n] = W[k1:n + 1, k1:n] - np.outer(Lp[k1:n + 1, t], Lp[k1:n, t])
        for i in range(k0, n + 1):                    # the panel's columns of L into W
            for j in range(k0, k1):
                if j <= i:
                    W[i, j] = Lp[i, j - k0]
    return np.tril(W[:n]), W[n]


@pytest.mark.parametrize("n,nb", [(1, 32), (2, 32), (7, 3), (33, 32), (70, 32), (100, 8)])
def test_panel_schedule_equals_column_factorization(n, nb):
    A = inputs.spd_matrix(n, 0.1, seed=800 + n)
    b = A @ inputs.solution(n, seed=801 + n)
    L, y = panel_schedule(A, b, nb)
    o = oracle.default()
    L0, st = o.chol_factor(A)
    assert st == 0
    assert np.array_equal(L, L0)                     # bit for bit
    assert np.array_equal(y, o.chol_forward(L0, b))
