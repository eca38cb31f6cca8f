"""Oracle for the dense Krylov solvers -- TEST INFRASTRUCTURE ONLY.

A plain FP64 CPU statement (in C, ``ls_oracle.c``) of what the GPU library
computes: conjugate gradient, restarted GMRES(m), Gaussian elimination with
partial pivoting, BF16 / FP8-e4m3 quantisation and the mixed-precision
refinement loop.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_1511_07207_gb300`` never does, and this package imports nothing from
it.  Arguments are numpy arrays; matrices are row-major.

The module-level functions use the oracle built from ``ls_oracle.c``;
:class:`Oracle` can also wrap another build of the same source (the tests
use that to check that planted mistakes are caught by the pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "ls_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libls_oracle.so")
_lock = threading.Lock()

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2


def compile_source(src: str, out: str) -> str:
    """gcc: plain C99, no FMA contraction, OpenMP for the row loops."""
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(SOURCE):
            compile_source(SOURCE, _LIB)
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _mat(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    assert A.ndim == 2
    return A


def _vec(v, n):
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    assert v.shape[0] == n
    return v


class Oracle:
    OK, NOT_CONVERGED, BREAKDOWN = OK, NOT_CONVERGED, BREAKDOWN

    def __init__(self, libpath: str):
        lib = ctypes.CDLL(libpath)
        d, i, l, f = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_float
        P = ctypes.c_void_p
        lib.or_gemv.argtypes = [i, i, P, l, P, P, i]
        lib.or_residual.argtypes = [i, P, l, P, P, P, i]
        lib.or_cg.argtypes = [i, P, l, P, P, d, i, i, i, P, P, P, P, P]
        lib.or_gmres.argtypes = [i, P, l, P, P, i, d, i, i, i, P, P, P, P, P, P, P]
        lib.or_bicgstab.argtypes = [i, P, l, P, P, d, i, i, i, P, P, P, P, P, P]
        lib.or_jacobi.argtypes = [i, P, l, P, P, d, i, i, i, P, P, P]
        lib.or_gauss_seidel.argtypes = [i, P, l, P, P, d, i, i, i, P, P, P]
        lib.or_block_cg.argtypes = [i, i, P, l, P, P, d, i, i, i, P, P]
        lib.or_block_cg_deflated.argtypes = [i, i, P, l, P, P, d, i, i, i, P, P, P]
        lib.or_block_gmres.argtypes = [i, i, P, l, P, P, i, d, i, i, i, i, P, P, P]
        lib.or_block_gmres_replacement.argtypes = [i, i, P]
        lib.or_block_gmres_replacement.restype = None
        lib.or_ge_solve.argtypes = [i, P, l, P, P]
        lib.or_ge_factor.argtypes = [i, P, l, P, P, P, P]
        lib.or_chol_factor.argtypes = [i, P, l, P]
        lib.or_chol_solve.argtypes = [i, P, l, P, P]
        lib.or_chol_forward.argtypes = [i, P, P, P]
        lib.or_chol_forward.restype = None
        for name in ("or_bf16_round", "or_e4m3_round"):
            getattr(lib, name).argtypes = [d]
            getattr(lib, name).restype = d
        lib.or_e4m3_decode.argtypes = [ctypes.c_uint8]
        lib.or_e4m3_decode.restype = d
        lib.or_bf16_decode.argtypes = [ctypes.c_uint16]
        lib.or_bf16_decode.restype = d
        lib.or_quant_bf16.argtypes = [i, i, P, l, P, l]
        lib.or_quant_fp8.argtypes = [i, i, P, l, P, l, P]
        lib.or_cg_f32.argtypes = [i, P, l, P, P, P, i, f, i]
        lib.or_mixed_cg.argtypes = [i, P, l, P, l, P, P, P, d, i, i, d, i, i, P, P, P, P, P]
        lib.or_max_threads.restype = i
        self.lib = lib

    def max_threads(self) -> int:
        return self.lib.or_max_threads()

    def gemv(self, A, x, nthreads=1):
        """y = A x (each row summed left to right)."""
        A = _mat(A)
        m, n = A.shape
        x = _vec(x, n)
        y = np.empty(m)
        assert self.lib.or_gemv(m, n, _p(A), n, _p(x), _p(y), nthreads) == 0
        return y

    def residual(self, A, b, x, nthreads=1):
        """r = b - A x."""
        A = _mat(A)
        n = A.shape[0]
        r = np.empty(n)
        assert self.lib.or_residual(n, _p(A), n, _p(_vec(b, n)), _p(_vec(x, n)), _p(r),
                                    nthreads) == 0
        return r

    def cg(self, A, b, rtol=1e-10, max_iter=None, x0=None, nthreads=1, history=False):
        """Conjugate gradient.  Returns dict(x, status, iters, rel_res[, res_hist, R, P])."""
        A = _mat(A)
        n = A.shape[0]
        b = _vec(b, n)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        x = np.zeros(n) if x0 is None else _vec(x0, n).copy()
        it, rr = ctypes.c_int(0), ctypes.c_double(0)
        rh = np.zeros(max_iter + 1) if history else None
        R = np.zeros((max_iter + 1, n)) if history else None
        P = np.zeros((max_iter + 1, n)) if history else None
        st = self.lib.or_cg(n, _p(A), n, _p(b), _p(x), rtol, max_iter, int(x0 is not None),
                            nthreads, ctypes.byref(it), ctypes.byref(rr), _p(rh), _p(R), _p(P))
        out = dict(x=x, status=st, iters=it.value, rel_res=rr.value)
        if history:
            k = it.value
            out.update(res_hist=rh[: k + 1], R=R[: k + 1], P=P[: k + 1])
        return out

    def jacobi(self, A, b, rtol=1e-10, max_iter=None, x0=None, nthreads=1, history=False):
        """Jacobi iteration.  Returns dict(x, status, iters, rel_res[, res_hist])."""
        return self._stationary(self.lib.or_jacobi, A, b, rtol, max_iter, x0, nthreads, history)

    def gauss_seidel(self, A, b, rtol=1e-10, max_iter=None, x0=None, nthreads=1, history=False):
        """Forward Gauss-Seidel.  Returns dict(x, status, iters, rel_res[, res_hist])."""
        return self._stationary(self.lib.or_gauss_seidel, A, b, rtol, max_iter, x0, nthreads, history)

    def block_cg(self, A, B, rtol=1e-10, max_iter=None, X0=None, nthreads=1):
        """O'Leary block CG on A X = B (B n x s).  Returns dict(X, status, iters, rel_res)."""
        A = _mat(A)
        n = A.shape[0]
        B = np.asarray(B, dtype=np.float64).reshape(n, -1)
        s = B.shape[1]
        Bc = np.asfortranarray(B)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        X = np.zeros((n, s), order="F") if X0 is None else np.asfortranarray(np.array(X0, dtype=np.float64).reshape(n, s))
        it, rr = ctypes.c_int(0), ctypes.c_double(0)
        st = self.lib.or_block_cg(n, s, _p(A), n, _p(Bc), _p(X), rtol, max_iter, int(X0 is not None),
                                  nthreads, ctypes.byref(it), ctypes.byref(rr))
        return dict(X=np.ascontiguousarray(X), status=st, iters=it.value, rel_res=rr.value)

    def block_cg_deflated(self, A, B, rtol=1e-10, max_iter=None, X0=None, nthreads=1):
        """Block CG with orthonormal, rank-revealed directions (dependent ones
        dropped).  Returns dict(X, status, iters, rel_res, rank)."""
        A = _mat(A)
        n = A.shape[0]
        B = np.asarray(B, dtype=np.float64).reshape(n, -1)
        s = B.shape[1]
        Bc = np.asfortranarray(B)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        X = np.zeros((n, s), order="F") if X0 is None else np.asfortranarray(np.array(X0, dtype=np.float64).reshape(n, s))
        it, rr, rk = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_int(0)
        st = self.lib.or_block_cg_deflated(n, s, _p(A), n, _p(Bc), _p(X), rtol, max_iter, int(X0 is not None),
                                           nthreads, ctypes.byref(it), ctypes.byref(rr), ctypes.byref(rk))
        return dict(X=np.ascontiguousarray(X), status=st, iters=it.value, rel_res=rr.value, rank=rk.value)

    def block_gmres(self, A, B, m=10, rtol=1e-10, max_iter=None, X0=None, deflate=1, nthreads=1):
        """Restarted block GMRES(m) on A X = B; deflate = 1 replaces the dependent
        columns of a cycle's starting block (0: they are a breakdown).
        Returns dict(X, status, iters, cycles, rel_res)."""
        A = _mat(A)
        n = A.shape[0]
        B = np.asarray(B, dtype=np.float64).reshape(n, -1)
        s = B.shape[1]
        Bc = np.asfortranarray(B)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        X = np.zeros((n, s), order="F") if X0 is None else np.asfortranarray(np.array(X0, dtype=np.float64).reshape(n, s))
        it, cy, rr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
        st = self.lib.or_block_gmres(n, s, _p(A), n, _p(Bc), _p(X), m, rtol, max_iter, int(X0 is not None),
                                     int(deflate), nthreads, ctypes.byref(it), ctypes.byref(cy), ctypes.byref(rr))
        return dict(X=np.ascontiguousarray(X), status=st, iters=it.value, cycles=cy.value, rel_res=rr.value)

    def block_gmres_replacement(self, n, c):
        """The vector that replaces dependent column c of a block GMRES
        starting block (n entries)."""
        z = np.zeros(max(n, 1))
        self.lib.or_block_gmres_replacement(n, c, _p(z))
        return z[:n]

    def _stationary(self, fn, A, b, rtol, max_iter, x0, nthreads, history):
        A = _mat(A)
        n = A.shape[0]
        b = _vec(b, n)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        x = np.zeros(n) if x0 is None else _vec(x0, n).copy()
        it, rr = ctypes.c_int(0), ctypes.c_double(0)
        rh = np.zeros(max_iter + 1) if history else None
        st = fn(n, _p(A), n, _p(b), _p(x), rtol, max_iter, int(x0 is not None),
                nthreads, ctypes.byref(it), ctypes.byref(rr), _p(rh))
        out = dict(x=x, status=st, iters=it.value, rel_res=rr.value)
        if history:
            out.update(res_hist=rh[: it.value])
        return out

    def bicgstab(self, A, b, rtol=1e-10, max_iter=None, x0=None, nthreads=1, trace=False):
        """BiCGSTAB.  Returns dict(x, status, iters, rel_res[, shs, rt, alphas])."""
        A = _mat(A)
        n = A.shape[0]
        b = _vec(b, n)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        x = np.zeros(n) if x0 is None else _vec(x0, n).copy()
        it, rr, steps = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_int(0)
        shs = np.zeros(max_iter + 1) if trace else None
        rt = np.zeros(max_iter + 1) if trace else None
        al = np.zeros(max_iter + 1) if trace else None
        st = self.lib.or_bicgstab(n, _p(A), n, _p(b), _p(x), rtol, max_iter, int(x0 is not None),
                                  nthreads, ctypes.byref(it), ctypes.byref(rr), _p(shs), _p(rt),
                                  _p(al), ctypes.byref(steps))
        out = dict(x=x, status=st, iters=it.value, rel_res=rr.value)
        if trace:
            out.update(shs=shs[: steps.value], rt=rt[: steps.value], alphas=al[: steps.value])
        return out

    def gmres(self, A, b, m=30, rtol=1e-10, max_iter=None, x0=None, nthreads=1,
              first_cycle=False):
        """Restarted GMRES(m).  Returns dict(x, status, iters, cycles, rel_res, est[, V, H, k])."""
        A = _mat(A)
        n = A.shape[0]
        b = _vec(b, n)
        max_iter = 10 * n + 10 if max_iter is None else max_iter
        x = np.zeros(n) if x0 is None else _vec(x0, n).copy()
        it, cy = ctypes.c_int(0), ctypes.c_int(0)
        rr, est = ctypes.c_double(0), ctypes.c_double(0)
        V = np.zeros((m + 1, n)) if first_cycle else None      # column-major n x (m+1)
        H = np.zeros((m, m + 1)) if first_cycle else None      # column-major (m+1) x m
        k1 = ctypes.c_int(0)
        st = self.lib.or_gmres(n, _p(A), n, _p(b), _p(x), m, rtol, max_iter,
                               int(x0 is not None), nthreads, ctypes.byref(it),
                               ctypes.byref(cy), ctypes.byref(rr), ctypes.byref(est),
                               _p(V), _p(H), ctypes.byref(k1))
        out = dict(x=x, status=st, iters=it.value, cycles=cy.value, rel_res=rr.value,
                   est=est.value)
        if first_cycle:
            out.update(V=V.T.copy(), H=H.T.copy(), k=k1.value)
        return out

    def ge_factor(self, A, b):
        """The elimination alone.  Returns (LU, ipiv, y, status): unit L below the
        diagonal and U on and above it (rows in pivoted order), the row swapped
        with row k at step k, and y = L^-1 P b."""
        A = _mat(A)
        n = A.shape[0]
        LU = np.zeros((n, n))
        ipiv = np.zeros(n, dtype=np.int32)
        y = np.zeros(n)
        st = self.lib.or_ge_factor(n, _p(A), n, _p(_vec(b, n)), _p(LU), _p(ipiv), _p(y))
        return LU, ipiv, y, st

    def chol_factor(self, A):
        """Cholesky factor L of an SPD A (lower triangular, zero above the
        diagonal).  Returns (L, status): status 2 when A is not SPD."""
        A = _mat(A)
        n = A.shape[0]
        L = np.zeros((n, n))
        st = self.lib.or_chol_factor(n, _p(A), n, _p(L))
        return L, st

    def chol_forward(self, L, b):
        """y = L^-1 b by forward substitution (sums in increasing column order)."""
        L = _mat(L)
        n = L.shape[0]
        y = np.zeros(n)
        self.lib.or_chol_forward(n, _p(L), _p(_vec(b, n)), _p(y))
        return y

    def chol_solve(self, A, b):
        """A x = b through A = L L^T.  Returns (x, status)."""
        A = _mat(A)
        n = A.shape[0]
        x = np.zeros(n)
        st = self.lib.or_chol_solve(n, _p(A), n, _p(_vec(b, n)), _p(x))
        return x, st

    def ge_solve(self, A, b):
        """Gaussian elimination with partial pivoting.  Returns (x, status)."""
        A = _mat(A)
        n = A.shape[0]
        x = np.zeros(n)
        st = self.lib.or_ge_solve(n, _p(A), n, _p(_vec(b, n)), _p(x))
        return x, st

    def bf16_round(self, d: float) -> float:
        return self.lib.or_bf16_round(float(d))

    def e4m3_round(self, d: float) -> float:
        return self.lib.or_e4m3_round(float(d))

    def e4m3_decode(self, c: int) -> float:
        return self.lib.or_e4m3_decode(int(c))

    def bf16_decode(self, c: int) -> float:
        return self.lib.or_bf16_decode(int(c))

    def quant_bf16(self, A):
        """BF16 codes (uint16, row-major) of A, round-to-nearest-even from FP64."""
        A = _mat(A)
        m, n = A.shape
        Q = np.zeros((m, n), dtype=np.uint16)
        assert self.lib.or_quant_bf16(m, n, _p(A), n, _p(Q), n) == 0
        return Q

    def quant_fp8(self, A):
        """FP8-e4m3 codes (uint8) and FP32 row scales of A."""
        A = _mat(A)
        m, n = A.shape
        Q = np.zeros((m, n), dtype=np.uint8)
        s = np.zeros(m, dtype=np.float32)
        assert self.lib.or_quant_fp8(m, n, _p(A), n, _p(Q), n, _p(s)) == 0
        return Q, s

    @staticmethod
    def decode_bf16(Q):
        """BF16 codes -> FP32 values (exact)."""
        return (np.asarray(Q, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)

    def decode_fp8(self, Q):
        """FP8-e4m3 codes -> FP32 values (exact), through the oracle's decoder."""
        table = np.array([self.e4m3_decode(c) for c in range(256)], dtype=np.float32)
        return table[np.asarray(Q, dtype=np.uint8)]

    def cg_f32(self, Af, rhs, iters, inner_rtol=0.0, scale=None, nthreads=1):
        """FP32 CG on the stored matrix (inner solver of the mixed path)."""
        Af = np.ascontiguousarray(Af, dtype=np.float32)
        n = Af.shape[0]
        rhs = np.ascontiguousarray(rhs, dtype=np.float32)
        z = np.zeros(n, dtype=np.float32)
        s = None if scale is None else np.ascontiguousarray(scale, dtype=np.float32)
        k = self.lib.or_cg_f32(n, _p(Af), n, _p(s), _p(rhs), _p(z), iters, inner_rtol,
                               nthreads)
        return z, k

    def mixed_cg(self, A, Af, b, scale=None, rtol=1e-10, max_outer=60, inner_iters=25,
                 inner_rtol=0.0, mode="fcg", nthreads=1, directions=False):
        """FP64 outer refinement (mode 'fcg' or 'ir') around FP32 inner CG on Af."""
        A = _mat(A)
        n = A.shape[0]
        Af = np.ascontiguousarray(Af, dtype=np.float32)
        s = None if scale is None else np.ascontiguousarray(scale, dtype=np.float32)
        x = np.zeros(n)
        o, i, rr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
        hist = np.zeros(max_outer + 2)
        P = np.zeros((max_outer + 1, n)) if directions else None
        st = self.lib.or_mixed_cg(n, _p(A), n, _p(Af), n, _p(s), _p(_vec(b, n)), _p(x), rtol,
                                  max_outer, inner_iters, inner_rtol,
                                  0 if mode == "fcg" else 1, nthreads, ctypes.byref(o),
                                  ctypes.byref(i), ctypes.byref(rr), _p(hist), _p(P))
        out = dict(x=x, status=st, outer=o.value, inner=i.value, rel_res=rr.value,
                   res_hist=hist[: o.value + 1])
        if directions:
            out["P"] = P
        return out


_default: Oracle | None = None


def default() -> Oracle:
    global _default
    if _default is None:
        path = build()
        with _lock:
            if _default is None:
                _default = Oracle(path)
    return _default


def __getattr__(name):
    # module-level access to the default oracle's methods: oracle.cg(...), ...
    if name.startswith("_"):
        raise AttributeError(name)
    return getattr(default(), name)
