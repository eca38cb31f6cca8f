"""Failure detection on the GPU without a fault: every on-device wait is
bounded.  A kernel waits on an mbarrier that nothing completes, and one CTA
waits at a grid barrier the other CTA never reaches; each gives up after the
limit (2 s), records the timeout, and the host reads LS_ERR_TIMEOUT.  The
same context then solves a system normally."""
import time

import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B
from paper_1511_07207_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_wait_gives_up_and_context_survives(ctx, gpu, which):
    t0 = time.time()
    assert B.ls_selftest_waits(ctx, which) == B.LS_ERR_TIMEOUT
    assert 1.5 < time.time() - t0 < 30.0
    n = 64
    A = inputs.spd_matrix(n, 0.1, seed=11)
    b = A @ inputs.solution(n, seed=11)
    x = torch.zeros(n, dtype=torch.float64, device=gpu)
    st, info = B.ls_cg_solve(ctx, torch.from_numpy(A).to(gpu), torch.from_numpy(b).to(gpu), x)
    assert st == B.LS_OK
    assert np.linalg.norm(A @ x.cpu().numpy() - b) <= 1e-10 * np.linalg.norm(b)
    assert B.ls_selftest_waits(ctx, 2) == B.LS_ERR_ARG
