"""The Python binding checks array shapes, layouts and dtypes before it
hands pointers to the C library (which reads exactly n elements from every
vector and rows x lda from every matrix), and raises instead of passing a
layout the library would misread.  CPU test: the arrays are host arrays and
the context is NULL, so a call that passes the checks reaches the library
and is refused there with LS_ERR_ARG."""
import numpy as np
import pytest
import torch

from paper_1511_07207_gb300 import binding as B

n = 6


def _sys():
    A = np.eye(n) * 2.0
    return A, np.ones(n), np.zeros(n)


@pytest.mark.parametrize("fn", [B.ls_cg_solve, B.ls_gmres_solve, B.ls_bicgstab_solve, B.ls_jacobi_solve,
                                B.ls_gauss_seidel_solve, B.ls_lu_solve])
def test_single_rhs_solves(fn):
    A, b, x = _sys()
    assert fn(None, A, b, x)[0] == B.LS_ERR_ARG                    # valid forms reach the library
    At = torch.from_numpy(A)
    assert fn(None, At, torch.from_numpy(b), torch.zeros(n, dtype=torch.float64))[0] == B.LS_ERR_ARG
    with pytest.raises(ValueError):
        fn(None, A, b[:-1], x)                                     # too short
    with pytest.raises(ValueError):
        fn(None, A, np.ones((n, 2))[:, 0], x)                      # strided view
    with pytest.raises(ValueError):
        fn(None, A[:, :-1], b[:-1], x[:-1])                        # not square
    with pytest.raises(ValueError):
        fn(None, np.asfortranarray(A + np.triu(np.ones((n, n)))), b, x)   # column-major A
    with pytest.raises(ValueError):
        fn(None, At.t(), torch.from_numpy(b), torch.zeros(n, dtype=torch.float64))   # transposed view
    with pytest.raises(TypeError):
        fn(None, A.astype(np.float32), b, x)


def test_block_solves():
    A = np.eye(n) * 2.0
    Bm = np.asfortranarray(np.ones((n, 3)))
    X = np.asfortranarray(np.zeros((n, 3)))
    for fn in (B.ls_block_cg_solve, B.ls_block_gmres_solve):
        assert fn(None, A, Bm, X)[0] == B.LS_ERR_ARG
        Xt = torch.zeros((3, n), dtype=torch.float64).t()          # columns contiguous
        assert fn(None, torch.from_numpy(A), torch.from_numpy(np.ascontiguousarray(Bm.T)).t(), Xt)[0] == B.LS_ERR_ARG
        with pytest.raises(ValueError):
            fn(None, A, Bm, np.ascontiguousarray(X))               # row-major X
        with pytest.raises(ValueError):
            fn(None, A, Bm, np.asfortranarray(np.zeros((n, 2))))   # shape mismatch


def test_lu_factor_outputs():
    A, b, _ = _sys()
    LU, y = np.zeros((n, n)), np.zeros(n)
    assert B.ls_lu_factor(None, A, b, LU, np.zeros(n, dtype=np.int32), y) == B.LS_ERR_ARG
    with pytest.raises(TypeError):
        B.ls_lu_factor(None, A, b, LU, np.zeros(n, dtype=np.int64), y)
    with pytest.raises(ValueError):
        B.ls_lu_factor(None, A, b, LU, np.zeros(n - 1, dtype=np.int32), y)
    with pytest.raises(ValueError):
        B.ls_lu_factor(None, A, b, np.zeros((n - 1, n)), np.zeros(n, dtype=np.int32), y)


def test_gemv_family():
    A = np.ones((4, 7))
    x, y = np.ones(7), np.zeros(4)
    assert B.ls_gemv(None, B.LS_F64, A, x, y) == B.LS_ERR_ARG
    with pytest.raises(ValueError):
        B.ls_gemv(None, B.LS_F64, A, np.ones(4), y)                # x must have cols elements
    with pytest.raises(ValueError):
        B.ls_gemv_timed(None, B.LS_F64, A, x, np.zeros(7), 1)
    Q = torch.zeros((4, 16), dtype=torch.int16)[:, :7]             # padded rows, as the tests pass it
    assert B.ls_quantize(None, B.LS_BF16_IR, A, Q) == B.LS_ERR_ARG
    with pytest.raises(ValueError):
        B.ls_quantize(None, B.LS_BF16_IR, A, torch.zeros((3, 7), dtype=torch.int16))
    pair = torch.zeros((8, 8), dtype=torch.float32)[:, :7]
    assert B.ls_split_f64(None, A, pair) == B.LS_ERR_ARG
    with pytest.raises(ValueError):
        B.ls_split_f64(None, A, torch.zeros((4, 8), dtype=torch.float32))   # hi rows only


def test_make_system():
    A = np.eye(n)
    Bm = np.asfortranarray(np.ones((n, 2)))
    s = B.make_system(B.LS_METHOD_CG, A, Bm, np.asfortranarray(np.zeros((n, 2))))
    assert s.n == n and s.nrhs == 2 and s.ldb == n and s.lda == n
    s = B.make_system(B.LS_METHOD_GMRES, A, np.ones(n), np.zeros(n))
    assert s.nrhs == 1 and s.ldb == n
    with pytest.raises(ValueError):
        B.make_system(B.LS_METHOD_CG, A, Bm, np.asfortranarray(np.zeros((n, 3))))
    with pytest.raises(ValueError):
        B.make_system(B.LS_METHOD_CG, A, np.ones((n, 2)), np.zeros((n, 2)))      # row-major blocks
    with pytest.raises(TypeError):
        B.make_system(B.LS_METHOD_CG, A.astype(np.float32), Bm, Bm.copy(order="F"))


def test_make_system_keeps_its_arrays_alive():
    """The descriptor holds raw pointers: it must keep the arrays it points to
    alive, or a temporary passed straight in would be freed (and its memory
    reused) before the solve."""
    import gc
    import weakref
    import numpy as np
    from paper_1511_07207_gb300 import binding as B
    A = np.eye(4)
    Bm = np.asfortranarray(np.ones((4, 2)))
    s = B.make_system(B.LS_METHOD_CG, A, Bm, np.asfortranarray(np.zeros((4, 2))))
    ref = weakref.ref(s._arrays[2])
    gc.collect()
    assert ref() is not None and s.X == s._arrays[2].ctypes.data
    del s
    gc.collect()
    assert ref() is None
