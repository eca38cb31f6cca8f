"""The seeded input recipes: reproducible bits, exact symmetry, spectra."""
import math

import numpy as np

from paper_1511_07207_gb300 import inputs


def test_reproducible_and_distinct():
    a = inputs.spd_matrix(64, 0.1, seed=0)
    b = inputs.spd_matrix(64, 0.1, seed=0)
    c = inputs.spd_matrix(64, 0.1, seed=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(inputs.solution(64, 3), inputs.solution(64, 3))


def test_spd_exactly_symmetric_with_expected_spectrum():
    n = 256
    for sigma in (0.1, 1e-3):
        A = inputs.spd_matrix(n, sigma, seed=2)
        assert np.array_equal(A, A.T)
        ev = np.linalg.eigvalsh(A)
        assert ev[0] >= sigma * (1 - 1e-9)
        assert ev[-1] <= 4.5 + sigma


def test_nonsym_spectrum_disk():
    n = 300
    A = inputs.nonsym_matrix(n, seed=4)
    ev = np.linalg.eigvals(A)
    assert np.max(np.abs(ev - 2.0)) <= 0.6
    R = inputs.restart_matrix(n, seed=4)
    ev = np.linalg.eigvals(R)
    assert np.max(np.abs(ev - 1.1)) <= 1.15


def test_solution_range():
    x = inputs.solution(1000, 0)
    assert x.min() >= -1 and x.max() <= 1 and abs(x.mean()) < 0.1
    X = inputs.solution(100, 0, nrhs=5)
    assert X.shape == (100, 5)


def test_batch_specs():
    specs = inputs.batch_specs(512, seed=0)
    ns = np.array([s.n for s in specs])
    assert len(specs) == 512 and ns.min() >= 64 and ns.max() <= 2048
    assert sum(s.kind == "spd" for s in specs) == 256
    assert all(1 <= s.nrhs <= 32 for s in specs)
    # log-uniform: median near the geometric mean of the range
    assert abs(math.log(np.median(ns)) - 0.5 * (math.log(64) + math.log(2048))) < 0.3
    assert len({s.seed for s in specs}) == 512


def test_serve_requests_poisson():
    reqs, pool = inputs.serve_requests(rate=2000.0, duration=1.0, seed=0)
    assert 1800 < len(reqs) < 2200
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean([r.spec.rtol == 1e-10 for r in reqs]) - 0.5) < 0.06
    assert len(pool) == 128 and all(128 <= p.n <= 8192 for p in pool)
