"""ls_gemv_noalloc: the matrix-vector product for callers that cannot allocate
device memory (a process whose memory is fully reserved by a pool or a
framework's caching allocator, or a latency-bound loop that must not pay for
cudaMalloc / cudaFree).  Its scratch lives in a static device array shared by
every call.

Each case makes two calls in a row with different shapes, to show that
nothing left in the shared array by the first call leaks into the second.
Every result is checked twice:
  * against the oracle's product (FP64: 2 gamma_n |A||x|; the FP32 pair:
    cols 2^-45 |A||x|; BF16 / FP8: the FP64 product of the decoded matrix
    within 2 gamma_{n+2}(FP32) |A||x|, as in the other GEMV tests);
  * against ls_gemv, the entry point with a context's allocated scratch: the
    same kernel with the same grid sums in the same order, so the two agree
    bit for bit.
Shapes with an odd FP64 column count take the plain-load kernel; shapes whose
rows are 16-byte aligned (contiguous torch tensors, even FP64 column counts,
column counts that are multiples of 8 for BF16 and 16 for FP8) take the TMA
kernel, whose matrix descriptor lives in the static array.

This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _gamma(n, u):
    return n * u / (1 - n * u)


def _two_calls(ctx, gpu, dtype, make, shapes):
    stream = torch.cuda.current_stream(gpu)
    for call, (rows, cols) in enumerate(shapes):
        rng = np.random.default_rng(100 + 10 * call + dtype)
        A_dev, scale, x, ref, bound = make(rng, rows, cols)
        odt = torch.float64 if dtype in (B.LS_F64, B.LS_F64_PAIR) else torch.float32
        xd = torch.from_numpy(x).to(gpu)
        y_ref = torch.full((rows,), np.nan, dtype=odt, device=gpu)
        y_na = torch.full((rows,), np.nan, dtype=odt, device=gpu)
        assert B.ls_gemv(ctx, dtype, A_dev, xd, y_ref, scale) == B.LS_OK
        assert B.ls_gemv_noalloc(dtype, A_dev, xd, y_na, scale, stream=stream) == B.LS_OK
        got = y_na.cpu().numpy()
        assert np.all(np.isfinite(got)), "call %d" % (call + 1)
        assert np.array_equal(got, y_ref.cpu().numpy()), "call %d differs from ls_gemv" % (call + 1)
        err = np.abs(got.astype(np.float64) - ref)
        assert np.all(err <= bound + 1e-300), "call %d outside the oracle bound" % (call + 1)


@pytest.mark.parametrize("shapes", [((1000, 1537), (3001, 257)),      # plain loads
                                    ((2048, 1024), (1000, 2048))])    # TMA
def test_noalloc_f64(ctx, gpu, oracle, shapes):
    def make(rng, rows, cols):
        A = rng.standard_normal((rows, cols))
        x = rng.standard_normal(cols)
        return (torch.from_numpy(A).to(gpu), None, x, oracle.gemv(A, x),
                2 * _gamma(cols, 2.0 ** -53) * (np.abs(A) @ np.abs(x)))
    _two_calls(ctx, gpu, B.LS_F64, make, shapes)


def test_noalloc_f64_pair(ctx, gpu, oracle):
    def make(rng, rows, cols):
        A = rng.standard_normal((rows, cols))
        x = rng.standard_normal(cols)
        ldp = (cols + 3) // 4 * 4
        pair = torch.full((2 * rows, ldp), np.nan, dtype=torch.float32, device=gpu)
        assert B.ls_split_f64(ctx, torch.from_numpy(A).to(gpu), pair[:, :cols]) == B.LS_OK
        return (pair[:rows, :cols], None, x, oracle.gemv(A, x),
                cols * 2.0 ** -45 * (np.abs(A) @ np.abs(x)))
    _two_calls(ctx, gpu, B.LS_F64_PAIR, make, [(1024, 2048), (777, 1001)])


@pytest.mark.parametrize("dtype", [B.LS_BF16_IR, B.LS_FP8_IR])
def test_noalloc_low_precision(ctx, gpu, oracle, dtype):
    def make(rng, rows, cols):
        A = rng.standard_normal((rows, cols))
        x = rng.standard_normal(cols).astype(np.float32)
        if dtype == B.LS_BF16_IR:
            codes = oracle.quant_bf16(A)
            Ah = oracle.decode_bf16(codes).astype(np.float64)
            Qd, sd = torch.from_numpy(codes.view(np.int16)).to(gpu), None
        else:
            codes, s = oracle.quant_fp8(A)
            Ah = oracle.decode_fp8(codes).astype(np.float64) * s[:, None].astype(np.float64)
            Qd, sd = torch.from_numpy(codes).to(gpu), torch.from_numpy(s).to(gpu)
        xf = x.astype(np.float64)
        return Qd, sd, x, Ah @ xf, 2 * _gamma(cols + 2, 2.0 ** -24) * (np.abs(Ah) @ np.abs(xf))
    _two_calls(ctx, gpu, dtype, make, [(2048, 4096), (513, 1000)])


def test_noalloc_rejects_bad_arguments(gpu):
    x = torch.zeros(8, dtype=torch.float64, device=gpu)
    A = torch.zeros((8, 8), dtype=torch.float64, device=gpu)
    lib = B.load()
    assert lib.ls_gemv_noalloc(B.LS_F64, 8, 8, B.ptr(A), 4, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
    assert lib.ls_gemv_noalloc(9, 8, 8, B.ptr(A), 8, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
    assert lib.ls_gemv_noalloc(B.LS_FP8_IR, 8, 8, B.ptr(A), 8, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
    # the FP32 pair needs 16-byte rows (lda a multiple of 4)
    assert lib.ls_gemv_noalloc(B.LS_F64_PAIR, 4, 6, B.ptr(A), 6, None, B.ptr(x), B.ptr(x), None) == B.LS_ERR_ARG
