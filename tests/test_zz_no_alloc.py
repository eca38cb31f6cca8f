"""ls_gemv_noalloc: the matrix-vector product for callers that cannot allocate
device memory (a process whose memory is fully reserved by a pool or a
framework's caching allocator, or a latency-bound loop that must not pay for
cudaMalloc / cudaFree).  Its scratch lives in a static device array shared by
every call, so two calls in a row must both match ls_gemv (the entry point
that uses a context's allocated scratch) within the FP64 product bound used
by the other GEMV tests; the second call uses another shape to show that
nothing left over from the first one leaks into it.

This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _bound(A, x):
    n = A.shape[1]
    u = 2.0 ** -53
    return 2 * (n * u / (1 - n * u)) * (np.abs(A) @ np.abs(x))


@pytest.mark.parametrize("shapes", [((1000, 1537), (3001, 257))])
def test_noalloc_matches_ls_gemv_twice(ctx, gpu, shapes):
    stream = torch.cuda.current_stream(gpu)
    for call, (rows, cols) in enumerate(shapes):
        rng = np.random.default_rng(100 + call)
        A = rng.standard_normal((rows, cols))
        x = rng.standard_normal(cols)
        Ad = torch.from_numpy(A).to(gpu)
        xd = torch.from_numpy(x).to(gpu)
        y_ref = torch.full((rows,), np.nan, dtype=torch.float64, device=gpu)
        y_na = torch.full((rows,), np.nan, dtype=torch.float64, device=gpu)
        assert B.ls_gemv(ctx, B.LS_F64, Ad, xd, y_ref) == B.LS_OK
        assert B.ls_gemv_noalloc(B.LS_F64, Ad, xd, y_na, stream=stream) == B.LS_OK
        a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.all(np.abs(a - b) <= _bound(A, x) + 1e-300), "call %d" % (call + 1)


def test_noalloc_rejects_bad_arguments(gpu):
    x = torch.zeros(8, dtype=torch.float64, device=gpu)
    A = torch.zeros((8, 8), dtype=torch.float64, device=gpu)
    lib = B.load()
    assert lib.ls_gemv_noalloc(B.LS_F64, 8, 8, B.ptr(A), 4, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
    assert lib.ls_gemv_noalloc(9, 8, 8, B.ptr(A), 8, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
    assert lib.ls_gemv_noalloc(B.LS_FP8_IR, 8, 8, B.ptr(A), 8, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
