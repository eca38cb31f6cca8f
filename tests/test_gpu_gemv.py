"""GPU parity of the matrix-vector product (K1 FP64, K2 BF16/FP8/FP32) and of
the quantisation of A, against the oracle, through the C ABI.

FP64: |y_gpu - y_oracle| <= 2 gamma_n |A| |x| elementwise (Higham's bound for
two summation orders, u = 2^-53).  FP64 through the FP32 pair (the solvers'
default): the split must equal fp32 rounding bit for bit, and the
double-single product stays within cols 2^-45 |A| |x| of the oracle (each
term carries errors of order 2^-48 |a x|, the low accumulator adds at most
one 2^-24 rounding of an O(2^-24) quantity per term).  Low precision: the stored codes must equal
the oracle's bit for bit; the product is compared with the FP64 product of the
oracle-decoded matrix within 2 gamma_n(FP32) |A| |x|.  Sizes span several
tiles with ragged row and column tails, padded leading dimensions, and odd
leading dimensions (which take the plain-load path instead of TMA).
"""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 0), (2, 3, 1), (31, 33, 0), (33, 257, 7), (255, 256, 0), (513, 1000, 8),
          (1000, 513, 1), (2049, 2047, 1), (300, 4100, 4), (4096, 4096, 0)]


def gamma(n, u):
    return n * u / (1 - n * u)


def _strided(rng, rows, cols, pad):
    full = rng.standard_normal((rows, cols + pad))
    return full, full[:, :cols]


@pytest.mark.parametrize("rows,cols,pad", SHAPES)
def test_gemv_f64(ctx, gpu, oracle, rows, cols, pad):
    rng = np.random.default_rng(rows * 7 + cols)
    full, A = _strided(rng, rows, cols, pad)
    x = rng.standard_normal(cols)
    Ad = torch.from_numpy(full).to(gpu)[:, :cols]
    xd = torch.from_numpy(x).to(gpu)
    yd = torch.full((rows,), np.nan, dtype=torch.float64, device=gpu)
    assert B.ls_gemv(ctx, B.LS_F64, Ad, xd, yd) == B.LS_OK
    y = yd.cpu().numpy()
    ref = oracle.gemv(np.ascontiguousarray(A), x)
    bound = 2 * gamma(cols, 2.0 ** -53) * (np.abs(A) @ np.abs(x))
    assert np.all(np.abs(y - ref) <= bound + 1e-300)


@pytest.mark.parametrize("rows,cols,pad", [(1, 1, 0), (31, 33, 3), (255, 256, 0), (513, 1000, 8),
                                          (2049, 2047, 1), (300, 4100, 4), (4096, 4096, 0)])
def test_gemv_f64_pair(ctx, gpu, oracle, rows, cols, pad):
    rng = np.random.default_rng(rows * 11 + cols)
    full, A = _strided(rng, rows, cols, pad)
    x = rng.standard_normal(cols)
    Ad = torch.from_numpy(full).to(gpu)[:, :cols]
    ldp = (cols + 3) // 4 * 4
    pair = torch.full((2 * rows, ldp), np.nan, dtype=torch.float32, device=gpu)
    assert B.ls_split_f64(ctx, Ad, pair[:, :cols]) == B.LS_OK
    hi = pair[:rows, :cols].cpu().numpy()
    lo = pair[rows:, :cols].cpu().numpy()
    assert np.array_equal(hi, A.astype(np.float32))
    assert np.array_equal(lo, (A - hi.astype(np.float64)).astype(np.float32))
    xd = torch.from_numpy(x).to(gpu)
    yd = torch.full((rows,), np.nan, dtype=torch.float64, device=gpu)
    assert B.ls_gemv(ctx, B.LS_F64_PAIR, pair[:rows, :cols], xd, yd) == B.LS_OK
    y = yd.cpu().numpy()
    ref = oracle.gemv(np.ascontiguousarray(A), x)
    bound = cols * 2.0 ** -45 * (np.abs(A) @ np.abs(x))
    assert np.all(np.abs(y - ref) <= bound + 1e-300)
    # and far closer than an FP32 product would be
    assert np.max(np.abs(y - ref) / (np.abs(A) @ np.abs(x))) < 1e-12


def test_gemv_deterministic(ctx, gpu):
    rng = np.random.default_rng(3)
    A = torch.from_numpy(rng.standard_normal((3000, 3001))).to(gpu)
    x = torch.from_numpy(rng.standard_normal(3001)).to(gpu)
    y1 = torch.empty(3000, dtype=torch.float64, device=gpu)
    y2 = torch.empty_like(y1)
    B.ls_gemv(ctx, B.LS_F64, A, x, y1)
    B.ls_gemv(ctx, B.LS_F64, A, x, y2)
    assert torch.equal(y1, y2)


def _quant(ctx, gpu, dtype, A):
    rows, cols = A.shape
    ldq = (cols + 15) // 16 * 16
    Ad = torch.from_numpy(A).to(gpu)
    tdt = {B.LS_BF16_IR: torch.int16, B.LS_FP8_IR: torch.uint8, B.LS_F32_IR: torch.float32}[dtype]
    Q = torch.zeros((rows, ldq), dtype=tdt, device=gpu)[:, :cols]
    s = torch.zeros(rows, dtype=torch.float32, device=gpu) if dtype == B.LS_FP8_IR else None
    assert B.ls_quantize(ctx, dtype, Ad, Q, s) == B.LS_OK
    return Q, s


@pytest.mark.parametrize("rows,cols", [(1, 1), (7, 33), (255, 513), (1024, 1000)])
def test_quantize_bitwise(ctx, gpu, oracle, rows, cols):
    rng = np.random.default_rng(rows + cols)
    A = rng.standard_normal((rows, cols)) * np.exp(rng.uniform(-8, 8, (rows, 1)))
    A[0, 0] = 0.0
    Q, _ = _quant(ctx, gpu, B.LS_BF16_IR, A)
    ref = oracle.quant_bf16(A)
    assert np.array_equal(Q.cpu().numpy().view(np.uint16), ref)
    Q, s = _quant(ctx, gpu, B.LS_FP8_IR, A)
    qref, sref = oracle.quant_fp8(A)
    assert np.array_equal(s.cpu().numpy(), sref)
    assert np.array_equal(Q.cpu().numpy(), qref)
    Q, _ = _quant(ctx, gpu, B.LS_F32_IR, A)
    assert np.array_equal(Q.cpu().numpy(), A.astype(np.float32))


@pytest.mark.parametrize("dtype", [B.LS_BF16_IR, B.LS_FP8_IR, B.LS_F32_IR])
@pytest.mark.parametrize("rows,cols", [(1, 5), (63, 300), (513, 1000), (2050, 4097)])
def test_gemv_lowp(ctx, gpu, oracle, dtype, rows, cols):
    rng = np.random.default_rng(rows * 3 + cols + dtype)
    A = rng.standard_normal((rows, cols))
    Q, s = _quant(ctx, gpu, dtype, A)
    x = rng.standard_normal(cols).astype(np.float32)
    y = torch.full((rows,), np.nan, dtype=torch.float32, device=gpu)
    assert B.ls_gemv(ctx, dtype, Q, torch.from_numpy(x).to(gpu), y, s) == B.LS_OK
    qh = Q.cpu().numpy()
    if dtype == B.LS_BF16_IR:
        Ah = oracle.decode_bf16(qh.view(np.uint16)).astype(np.float64)
    elif dtype == B.LS_FP8_IR:
        Ah = oracle.decode_fp8(qh).astype(np.float64) * s.cpu().numpy()[:, None].astype(np.float64)
    else:
        Ah = qh.astype(np.float64)
    ref = Ah @ x.astype(np.float64)
    bound = 2 * gamma(cols + 2, 2.0 ** -24) * (np.abs(Ah) @ np.abs(x.astype(np.float64)))
    assert np.all(np.abs(y.cpu().numpy().astype(np.float64) - ref) <= bound + 1e-30)


def _split_edge_values(rng, count):
    """Random bit patterns, random fractions at every binary exponent from
    -80 to 130, rounding ties and carries of the 29 dropped bits, and
    special values (zeros, subnormals, overflow to infinity, infinities, NaN)."""
    words = [rng.integers(0, 2 ** 63, size=count // 3, dtype=np.uint64) * np.uint64(2)
             + rng.integers(0, 2, size=count // 3, dtype=np.uint64)]
    E = rng.integers(-80, 131, size=count // 3).astype(np.uint64)
    frac = rng.integers(0, 2 ** 52, size=count // 3, dtype=np.uint64)
    sign = rng.integers(0, 2, size=count // 3, dtype=np.uint64)
    words.append((sign << np.uint64(63)) | ((E + np.uint64(1023)) << np.uint64(52)) | frac)
    ties = []
    for e in range(-80, 131):
        for keep in (0, 1, 2, 3, 0x7FFFFE, 0x7FFFFF):
            for R in (0, 1, (1 << 28) - 1, 1 << 28, (1 << 28) + 1, (1 << 29) - 1):
                for s in (0, 1):
                    ties.append((s << 63) | ((e + 1023) << 52) | (keep << 29) | R)
    words.append(np.array(ties, dtype=np.uint64))
    v = np.concatenate(words).view(np.float64)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300, 1e300,
                        3.4028235677973366e38, -3.4028235677973366e38, np.inf, -np.inf, np.nan, 1.0 / 3.0])
    return np.concatenate([v, special])


@pytest.mark.parametrize("cols,pad", [(1032, 0), (1029, 0), (1031, 1)])
def test_split_edge_values_bit_exact(ctx, gpu, cols, pad):
    """The split's hi and lo equal fp32(a) and fp32(a - hi) bit for bit on every
    input class, through the 16-byte path (even leading dimension) and the
    element path (odd leading dimension)."""
    rng = np.random.default_rng(cols)
    vals = _split_edge_values(rng, 150000)
    rows = -(-vals.size // cols)
    full = np.zeros((rows, cols + pad))
    flat = np.zeros(rows * cols)
    flat[:vals.size] = vals
    full[:, :cols] = flat.reshape(rows, cols)
    A = full[:, :cols]
    Ad = torch.from_numpy(full).to(gpu)[:, :cols]
    ldp = (cols + 3) // 4 * 4
    pair = torch.full((2 * rows, ldp), np.nan, dtype=torch.float32, device=gpu)
    assert B.ls_split_f64(ctx, Ad, pair[:, :cols]) == B.LS_OK
    hi = pair[:rows, :cols].cpu().numpy()
    lo = pair[rows:, :cols].cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        ref_hi = A.astype(np.float32)
        ref_lo = (A - ref_hi.astype(np.float64)).astype(np.float32)
    for got, ref in ((hi, ref_hi), (lo, ref_lo)):
        both_nan = np.isnan(got) & np.isnan(ref)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        assert np.array_equal(got.view(np.uint32)[~both_nan], ref.view(np.uint32)[~both_nan])
