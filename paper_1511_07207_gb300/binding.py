"""Thin Python binding of the C ABI in ``include/ls.h`` (ctypes).

The functions keep the C names and only marshal arguments: numpy arrays
(host memory) and torch tensors (host or CUDA memory) are turned into
pointers, sizes and leading dimensions; every step of a solve runs in the
CUDA library.  There is no CPU fallback: if the library cannot be loaded the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

LS_OK, LS_NOT_CONVERGED, LS_BREAKDOWN = 0, 1, 2
LS_ERR_ARG, LS_ERR_NOMEM, LS_ERR_CUDA, LS_ERR_TIMEOUT = -1, -2, -3, -4
LS_ERR_BUSY, LS_ERR_NAN, LS_ERR_UNSUPPORTED = -5, -6, -7
LS_METHOD_CG, LS_METHOD_GMRES, LS_METHOD_BICGSTAB, LS_METHOD_JACOBI, LS_METHOD_GAUSS_SEIDEL = 0, 1, 2, 3, 4
LS_METHOD_BLOCK_CG, LS_BLOCK_CG_MAX_S = 5, 16
LS_METHOD_BLOCK_GMRES, LS_BLOCK_GMRES_MAX_MS = 6, 256
LS_METHOD_LU = 7
LS_METHOD_CHOLESKY = 8
LS_F64, LS_BF16_IR, LS_FP8_IR, LS_F32_IR = 0, 1, 2, 3
LS_F64_PAIR = 4
LS_REFINE_FCG, LS_REFINE_IR = 0, 1
LS_MAX_RESTART = 128
LS_BATCH_MAX_N, LS_BATCH_MAX_RHS = 8192, 32
LS_TUNE_QUICK = 1

# every symbol declared in include/ls.h
ABI_FUNCTIONS = (
    "ls_opts_default", "ls_create", "ls_destroy", "ls_workspace_size", "ls_set_workspace",
    "ls_cg_solve", "ls_gmres_solve", "ls_bicgstab_solve", "ls_jacobi_solve", "ls_gauss_seidel_solve", "ls_block_cg_solve", "ls_block_gmres_solve", "ls_lu_solve", "ls_lu_factor", "ls_batch_solve", "ls_server_start", "ls_server_submit",
    "ls_server_poll", "ls_server_stop", "ls_gemv", "ls_gemv_timed", "ls_gemv_noalloc",
    "ls_quantize", "ls_split_f64", "ls_kernel_launches", "ls_strerror", "ls_selftest_waits",
    "ls_autotune", "ls_tune_load", "ls_tune_reset", "ls_tune_lookup", "ls_chol_solve", "ls_chol_factor",
)


class ls_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int), ("restart", ctypes.c_int),
                ("precision", ctypes.c_int), ("refine", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("x0_given", ctypes.c_int), ("reorth", ctypes.c_int), ("f64_matvec", ctypes.c_int),
                ("deflate", ctypes.c_int), ("fused", ctypes.c_int)]


class ls_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("bytes_moved", ctypes.c_double),
                ("launches", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ls_system(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("n", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("opts", ls_opts)]


class ls_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("step_iters", ctypes.c_int), ("queue_capacity", ctypes.c_int),
                ("merge_rhs", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the CUDA library (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.ls_opts_default.argtypes = [ctypes.POINTER(ls_opts)]
        lib.ls_create.argtypes = [ctypes.POINTER(P), I, P]
        lib.ls_destroy.argtypes = [P]
        lib.ls_workspace_size.argtypes = [P, I, I, I, ctypes.POINTER(ls_opts), I,
                                          ctypes.POINTER(ctypes.c_size_t)]
        lib.ls_set_workspace.argtypes = [P, P, ctypes.c_size_t]
        for fn in (lib.ls_cg_solve, lib.ls_gmres_solve, lib.ls_bicgstab_solve, lib.ls_jacobi_solve,
               lib.ls_gauss_seidel_solve, lib.ls_lu_solve, lib.ls_chol_solve):
            fn.argtypes = [P, I, P, I64, P, P, ctypes.POINTER(ls_opts), ctypes.POINTER(ls_info)]
        for fn in (lib.ls_block_cg_solve, lib.ls_block_gmres_solve):
            fn.argtypes = [P, I, I, P, I64, P, I64, P, I64, ctypes.POINTER(ls_opts), ctypes.POINTER(ls_info)]
        lib.ls_lu_factor.argtypes = [P, I, P, I64, P, P, I64, P, P]
        lib.ls_chol_factor.argtypes = [P, I, P, I64, P, P, I64, P, ctypes.POINTER(I)]
        lib.ls_batch_solve.argtypes = [P, I, ctypes.POINTER(ls_system), ctypes.POINTER(ls_info)]
        lib.ls_server_start.argtypes = [P, ctypes.POINTER(ls_server_cfg), ctypes.POINTER(P)]
        lib.ls_server_submit.argtypes = [P, ctypes.POINTER(ls_system),
                                         ctypes.POINTER(ctypes.c_uint64)]
        lib.ls_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(I),
                                       ctypes.POINTER(ls_info)]
        lib.ls_server_stop.argtypes = [P]
        lib.ls_gemv.argtypes = [P, I, I, I, P, I64, P, P, P]
        lib.ls_gemv_timed.argtypes = [P, I, I, I, P, I64, P, P, P, I,
                                      ctypes.POINTER(ctypes.c_double)]
        lib.ls_gemv_noalloc.argtypes = [I, I, I, P, I64, P, P, P, P]
        lib.ls_quantize.argtypes = [P, I, I, I, P, I64, P, I64, P]
        lib.ls_split_f64.argtypes = [P, I, I, P, I64, P, I64]
        lib.ls_kernel_launches.argtypes = [P]
        lib.ls_selftest_waits.argtypes = [P, I]
        lib.ls_autotune.argtypes = [P, ctypes.c_char_p, I]
        lib.ls_tune_load.argtypes = [ctypes.c_char_p]
        lib.ls_tune_reset.argtypes = []
        lib.ls_tune_lookup.argtypes = [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.ls_kernel_launches.restype = ctypes.c_longlong
        lib.ls_strerror.argtypes = [I]
        lib.ls_strerror.restype = ctypes.c_char_p
        _lib = lib
        return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _itemsize(a):
    return a.element_size() if _is_torch(a) else a.itemsize


def lead_dim(a) -> int:
    """Leading dimension (elements) of a row-major 2-D array; rows must be
    unit-stride (ValueError otherwise)."""
    if _is_torch(a):
        if a.dim() != 2 or (a.shape[1] > 1 and a.stride(1) != 1):
            raise ValueError("a row-major 2-D array with unit column stride is required")
        return a.stride(0)
    if a.ndim != 2 or (a.shape[1] > 1 and a.strides[1] != a.itemsize):
        raise ValueError("a row-major 2-D array with unit column stride is required")
    return a.strides[0] // a.itemsize


def col_lead_dim(a) -> int:
    """Leading dimension of a column-major n x k block (column j at a + j*ld).
    A single column has no meaningful column stride (frameworks may report
    any value for a size-1 dimension), so its leading dimension is n."""
    if _is_torch(a):
        if a.dim() == 1 or a.shape[1] == 1:
            return a.shape[0]
        if a.stride(0) != 1:
            raise ValueError("a column-major block with unit row stride is required")
        return a.stride(1)
    if a.ndim == 1 or a.shape[1] == 1:
        return a.shape[0]
    if a.strides[0] != a.itemsize:
        raise ValueError("a column-major block with unit row stride is required")
    return a.strides[1] // a.itemsize


def make_opts(**kw) -> ls_opts:
    o = ls_opts()
    load().ls_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    return o


def _check_f64(*arrs):
    for a in arrs:
        if a is None:
            continue
        dt = str(a.dtype)
        if dt not in ("float64", "torch.float64"):
            raise TypeError("FP64 arrays required, got %s" % dt)


def _numel(a):
    return a.numel() if _is_torch(a) else a.size


def _check_vec(v, n, name):
    """v must hold n elements contiguously (the library reads v[0 .. n-1])."""
    if v is None:
        raise ValueError("%s is required" % name)
    contig = v.is_contiguous() if _is_torch(v) else v.flags["C_CONTIGUOUS"]
    if _numel(v) != n or not (contig or n <= 1):
        raise ValueError("%s: %d contiguous elements required, got shape %s" % (name, n, tuple(v.shape)))


def _check_square(A):
    if len(A.shape) != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be n x n, got shape %s" % (tuple(A.shape),))
    return A.shape[0]


# ---------------------------------------------------------------------------
# ABI functions (same names as include/ls.h)
# ---------------------------------------------------------------------------

def ls_create(device: int = 0, stream=None):
    """Returns an opaque context handle.  `stream` is a cudaStream_t (int), a
    torch.cuda.Stream, or None for the default stream."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    st = load().ls_create(ctypes.byref(h), device, stream)
    if st != LS_OK:
        raise RuntimeError("ls_create failed: %s" % ls_strerror(st))
    return h


def ls_destroy(ctx):
    return load().ls_destroy(ctx)


def ls_strerror(status: int) -> str:
    return load().ls_strerror(status).decode()


def ls_kernel_launches(ctx) -> int:
    return load().ls_kernel_launches(ctx)


def ls_workspace_size(ctx, method, n, nrhs=1, opts=None, a_on_device=True) -> int:
    b = ctypes.c_size_t(0)
    st = load().ls_workspace_size(ctx, method, n, nrhs, ctypes.byref(opts) if opts else None,
                                  int(a_on_device), ctypes.byref(b))
    if st != LS_OK:
        raise RuntimeError(ls_strerror(st))
    return b.value


def ls_set_workspace(ctx, buf=None, nbytes=0):
    return load().ls_set_workspace(ctx, ptr(buf), nbytes)


def _solve(fn, ctx, A, b, x, opts):
    _check_f64(A, b, x)
    n = _check_square(A)
    _check_vec(b, n, "b")
    _check_vec(x, n, "x")
    info = ls_info()
    o = opts if opts is not None else make_opts()
    st = fn(ctx, n, ptr(A), lead_dim(A), ptr(b), ptr(x), ctypes.byref(o), ctypes.byref(info))
    return st, info.as_dict()


def ls_cg_solve(ctx, A, b, x, opts=None):
    """CG on A x = b; A (n x n row-major), b, x FP64 (host or device).  x is
    written in place.  Returns (status, info dict)."""
    return _solve(load().ls_cg_solve, ctx, A, b, x, opts)


def ls_gmres_solve(ctx, A, b, x, opts=None):
    """Restarted GMRES(m) on A x = b; see ls_cg_solve."""
    return _solve(load().ls_gmres_solve, ctx, A, b, x, opts)


def ls_bicgstab_solve(ctx, A, b, x, opts=None):
    """BiCGSTAB on A x = b; see ls_cg_solve."""
    return _solve(load().ls_bicgstab_solve, ctx, A, b, x, opts)


def ls_jacobi_solve(ctx, A, b, x, opts=None):
    """Jacobi iteration on A x = b; see ls_cg_solve."""
    return _solve(load().ls_jacobi_solve, ctx, A, b, x, opts)


def ls_gauss_seidel_solve(ctx, A, b, x, opts=None):
    """Forward Gauss-Seidel on A x = b; see ls_cg_solve."""
    return _solve(load().ls_gauss_seidel_solve, ctx, A, b, x, opts)


def ls_gemv(ctx, dtype, A, x, y, scale=None):
    """y = A x on the device (see ls.h for the per-format types)."""
    rows, cols = A.shape
    _check_vec(x, cols, "x")
    _check_vec(y, rows, "y")
    if scale is not None:
        _check_vec(scale, rows, "scale")
    return load().ls_gemv(ctx, dtype, rows, cols, ptr(A), lead_dim(A), ptr(scale), ptr(x), ptr(y))


def ls_gemv_timed(ctx, dtype, A, x, y, reps, scale=None):
    """Mean device ms of one y = A x launch over `reps` back-to-back launches."""
    rows, cols = A.shape
    _check_vec(x, cols, "x")
    _check_vec(y, rows, "y")
    if scale is not None:
        _check_vec(scale, rows, "scale")
    ms = ctypes.c_double(0)
    st = load().ls_gemv_timed(ctx, dtype, rows, cols, ptr(A), lead_dim(A), ptr(scale), ptr(x),
                              ptr(y), reps, ctypes.byref(ms))
    return st, ms.value


def ls_gemv_noalloc(dtype, A, x, y, scale=None, stream=None):
    """y = A x with no device allocation and no context (see ls.h): for callers
    that cannot allocate device memory.  Runs on `stream` (a cudaStream_t int,
    a torch.cuda.Stream, or None) on the current device."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    rows, cols = A.shape
    _check_vec(x, cols, "x")
    _check_vec(y, rows, "y")
    if scale is not None:
        _check_vec(scale, rows, "scale")
    return load().ls_gemv_noalloc(dtype, rows, cols, ptr(A), lead_dim(A), ptr(scale), ptr(x),
                                  ptr(y), stream)


def ls_quantize(ctx, dtype, A, Q, scale=None):
    """Quantise FP64 A (device) into Q (device) [and FP32 row scales]."""
    rows, cols = A.shape
    if Q.shape[0] != rows or Q.shape[1] < cols:
        raise ValueError("Q must have %d rows and at least %d columns" % (rows, cols))
    if scale is not None:
        _check_vec(scale, rows, "scale")
    return load().ls_quantize(ctx, dtype, rows, cols, ptr(A), lead_dim(A), ptr(Q), lead_dim(Q),
                              ptr(scale))


def ls_split_f64(ctx, A, pair):
    """Split FP64 A (device, rows x cols) into the FP32 pair `pair` (device,
    2 rows x ldp floats: hi rows, then lo rows)."""
    rows, cols = A.shape
    if pair.shape[0] != 2 * rows or pair.shape[1] < cols:
        raise ValueError("pair must have %d rows and at least %d columns" % (2 * rows, cols))
    return load().ls_split_f64(ctx, rows, cols, ptr(A), lead_dim(A), ptr(pair), lead_dim(pair))


def make_system(method, A, B, X, opts=None) -> ls_system:
    """One system of a batch or a server request: A (n x n row-major), B and X
    n-vectors or n x k column-major blocks of the same shape, all FP64.  The
    descriptor holds raw pointers; it also keeps references to A, B and X, so
    the arrays live at least as long as the descriptor does (an expression
    such as ``torch.from_numpy(a).to(dev)`` passed straight in would
    otherwise be freed, and its memory reused, before the solve)."""
    _check_f64(A, B, X)
    n = _check_square(A)
    if B.shape[0] != n or tuple(X.shape) != tuple(B.shape):
        raise ValueError("B and X must be n-vectors or n x k blocks of the same shape")
    s = ls_system()
    s.method = method
    s.n = n
    s.nrhs = 1 if B.ndim == 1 else B.shape[1]
    s.A, s.lda = ptr(A), lead_dim(A)
    s.B, s.ldb = ptr(B), col_lead_dim(B)
    s.X, s.ldx = ptr(X), col_lead_dim(X)
    s.opts = opts if opts is not None else make_opts()
    s._arrays = (A, B, X)
    return s


def ls_block_cg_solve(ctx, A, B, X, opts=None):
    """Block CG on A X = B.  A (n x n row-major); B and X n x s blocks stored
    column by column (numpy Fortran order, or a torch tensor whose columns are
    contiguous, e.g. the transpose of a contiguous s x n tensor).  X is
    written in place.  Returns (status, info dict)."""
    _check_f64(A, B, X)
    n = _check_square(A)
    if B.shape[0] != n or tuple(X.shape) != tuple(B.shape):
        raise ValueError("B and X must be n x s blocks of the same shape")
    info = ls_info()
    o = opts if opts is not None else make_opts()
    st = load().ls_block_cg_solve(ctx, n, B.shape[1], ptr(A), lead_dim(A), ptr(B), col_lead_dim(B), ptr(X),
                                  col_lead_dim(X), ctypes.byref(o), ctypes.byref(info))
    return st, info.as_dict()


def ls_block_gmres_solve(ctx, A, B, X, opts=None):
    """Restarted block GMRES(m) on A X = B (m = opts.restart block steps);
    B and X as for ls_block_cg_solve.  Returns (status, info dict)."""
    _check_f64(A, B, X)
    n = _check_square(A)
    if B.shape[0] != n or tuple(X.shape) != tuple(B.shape):
        raise ValueError("B and X must be n x s blocks of the same shape")
    info = ls_info()
    o = opts if opts is not None else make_opts()
    st = load().ls_block_gmres_solve(ctx, n, B.shape[1], ptr(A), lead_dim(A), ptr(B), col_lead_dim(B), ptr(X),
                                     col_lead_dim(X), ctypes.byref(o), ctypes.byref(info))
    return st, info.as_dict()


def ls_lu_solve(ctx, A, b, x, opts=None):
    """The direct method: LU with partial pivoting, then U x = y; see ls_cg_solve."""
    return _solve(load().ls_lu_solve, ctx, A, b, x, opts)


def ls_lu_factor(ctx, A, b, LU, ipiv, y):
    """The factorization alone into LU (n x n row-major), ipiv (int32), y.  Returns the status."""
    _check_f64(A, b, LU, y)
    n = _check_square(A)
    _check_vec(b, n, "b")
    _check_vec(y, n, "y")
    _check_vec(ipiv, n, "ipiv")
    if str(ipiv.dtype) not in ("int32", "torch.int32"):
        raise TypeError("ipiv must be int32, got %s" % ipiv.dtype)
    if LU.shape[0] != n or LU.shape[1] < n:
        raise ValueError("LU must be n x n")
    return load().ls_lu_factor(ctx, n, ptr(A), lead_dim(A), ptr(b), ptr(LU), lead_dim(LU), ptr(ipiv), ptr(y))


def ls_chol_solve(ctx, A, b, x, opts=None):
    """The direct method for SPD A: A = L L^T, then L y = b, L^T x = y; see ls_cg_solve."""
    return _solve(load().ls_chol_solve, ctx, A, b, x, opts)


def ls_chol_factor(ctx, A, b, L, y):
    """The Cholesky factorization alone into L (n x n row-major, zeros above the
    diagonal) and y = L^-1 b.  Returns (status, step): step is the failing
    step on LS_BREAKDOWN, else -1."""
    _check_f64(A, b, L, y)
    n = _check_square(A)
    _check_vec(b, n, "b")
    _check_vec(y, n, "y")
    if L.shape[0] != n or L.shape[1] < n:
        raise ValueError("L must be n x n")
    step = ctypes.c_int(-1)
    st = load().ls_chol_factor(ctx, n, ptr(A), lead_dim(A), ptr(b), ptr(L), lead_dim(L), ptr(y),
                               ctypes.byref(step))
    return st, step.value


def ls_batch_solve(ctx, systems):
    """systems: list of ls_system (from make_system, which keeps their arrays
    alive).  Returns (status, [info dict])."""
    arr = (ls_system * len(systems))(*systems)
    infos = (ls_info * len(systems))()
    st = load().ls_batch_solve(ctx, len(systems), arr, infos)
    return st, [i.as_dict() for i in infos]


def ls_autotune(ctx, path=None, flags=0):
    """Time the batched engine's tile-shape candidates; write the JSON cache to
    `path` (str or None) and use the choices in this process."""
    return load().ls_autotune(ctx, path.encode() if path else None, flags)


def ls_tune_load(path):
    return load().ls_tune_load(path.encode())


def ls_tune_reset():
    return load().ls_tune_reset()


def ls_tune_lookup(n, nrhs, num_sms):
    """(status, ks32, tensor_cores) for an n x n system with nrhs columns."""
    ks, tc = ctypes.c_int(0), ctypes.c_int(0)
    st = load().ls_tune_lookup(n, nrhs, num_sms, ctypes.byref(ks), ctypes.byref(tc))
    return st, ks.value, tc.value


def ls_server_start(ctx, hbm_budget_bytes, max_slots=64, step_iters=8, queue_capacity=1 << 16,
                    merge_rhs=1):
    cfg = ls_server_cfg(hbm_budget_bytes, max_slots, step_iters, queue_capacity, merge_rhs)
    h = ctypes.c_void_p()
    st = load().ls_server_start(ctx, ctypes.byref(cfg), ctypes.byref(h))
    if st != LS_OK:
        raise RuntimeError("ls_server_start failed: %s" % ls_strerror(st))
    return h


def ls_server_submit(srv, system: ls_system):
    t = ctypes.c_uint64(0)
    st = load().ls_server_submit(srv, ctypes.byref(system), ctypes.byref(t))
    return st, t.value


def ls_server_poll(srv, ticket):
    done = ctypes.c_int(0)
    info = ls_info()
    st = load().ls_server_poll(srv, ticket, ctypes.byref(done), ctypes.byref(info))
    return st, bool(done.value), info.as_dict()


def ls_server_stop(srv):
    return load().ls_server_stop(srv)


def ls_selftest_waits(ctx, which):
    """Run the self-test of the bounded waits (0: mbarrier, 1: grid barrier);
    LS_ERR_TIMEOUT is the expected result."""
    return load().ls_selftest_waits(ctx, which)
