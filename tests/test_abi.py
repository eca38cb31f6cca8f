"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/ls.h; host-only calls work without a GPU (CPU test)."""
import ctypes
import os
import re

from paper_1511_07207_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(binding.ABI_FUNCTIONS) == _declared()


def test_library_exports_every_symbol(lslib):
    for name in _declared():
        assert hasattr(lslib, name), name
        assert ctypes.cast(getattr(lslib, name), ctypes.c_void_p).value


def test_host_only_calls(lslib):
    o = binding.make_opts()
    assert o.rtol == 1e-10 and o.restart == 30 and o.inner_iters == 25
    assert o.precision == binding.LS_F64 and o.refine == binding.LS_REFINE_FCG
    assert o.deflate == 1 and o.fused == 1 and o.f64_matvec == 0
    assert binding.ls_strerror(binding.LS_OK) == "converged"
    assert "argument" in binding.ls_strerror(binding.LS_ERR_ARG)
    assert lslib.ls_opts_default(None) == binding.LS_ERR_ARG
    # no context -> argument errors, never a crash
    info = binding.ls_info()
    assert lslib.ls_cg_solve(None, 4, None, 4, None, None, None, ctypes.byref(info)) == binding.LS_ERR_ARG
    assert lslib.ls_destroy(None) == binding.LS_OK


def test_create_without_gpu_fails_cleanly(lslib):
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    st = lslib.ls_create(ctypes.byref(h), 0, None)
    assert st in (binding.LS_ERR_CUDA, binding.LS_ERR_UNSUPPORTED)
    assert not h.value


def _null_context_calls(lib):
    """Every entry that takes a context (or a server), called with NULL and
    otherwise plausible arguments."""
    info, o = binding.ls_info(), binding.make_opts()
    buf = (ctypes.c_double * 16)()
    ib = (ctypes.c_int * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    pi = ctypes.cast(ib, ctypes.c_void_p)
    oi = (ctypes.byref(o), ctypes.byref(info))
    return {
        "ls_workspace_size": lambda: lib.ls_workspace_size(None, 1, 4, 1, ctypes.byref(o), 0,
                                                           ctypes.byref(ctypes.c_size_t())),
        "ls_set_workspace": lambda: lib.ls_set_workspace(None, p, 128),
        "ls_cg_solve": lambda: lib.ls_cg_solve(None, 4, p, 4, p, p, *oi),
        "ls_gmres_solve": lambda: lib.ls_gmres_solve(None, 4, p, 4, p, p, *oi),
        "ls_bicgstab_solve": lambda: lib.ls_bicgstab_solve(None, 4, p, 4, p, p, *oi),
        "ls_jacobi_solve": lambda: lib.ls_jacobi_solve(None, 4, p, 4, p, p, *oi),
        "ls_gauss_seidel_solve": lambda: lib.ls_gauss_seidel_solve(None, 4, p, 4, p, p, *oi),
        "ls_lu_solve": lambda: lib.ls_lu_solve(None, 4, p, 4, p, p, *oi),
        "ls_chol_solve": lambda: lib.ls_chol_solve(None, 4, p, 4, p, p, *oi),
        "ls_chol_factor": lambda: lib.ls_chol_factor(None, 2, p, 2, p, p, 2, p, None),
        "ls_block_cg_solve": lambda: lib.ls_block_cg_solve(None, 2, 2, p, 2, p, 2, p, 2, *oi),
        "ls_block_gmres_solve": lambda: lib.ls_block_gmres_solve(None, 2, 2, p, 2, p, 2, p, 2, *oi),
        "ls_lu_factor": lambda: lib.ls_lu_factor(None, 2, p, 2, p, p, 2, pi, p),
        "ls_batch_solve": lambda: lib.ls_batch_solve(None, 1, ctypes.byref(binding.ls_system()),
                                                     ctypes.byref(info)),
        "ls_server_start": lambda: lib.ls_server_start(None, ctypes.byref(binding.ls_server_cfg()),
                                                       ctypes.byref(ctypes.c_void_p())),
        "ls_server_submit": lambda: lib.ls_server_submit(None, ctypes.byref(binding.ls_system()),
                                                         ctypes.byref(ctypes.c_uint64())),
        "ls_server_poll": lambda: lib.ls_server_poll(None, 1, ctypes.byref(ctypes.c_int()), ctypes.byref(info)),
        "ls_server_stop": lambda: lib.ls_server_stop(None),
        "ls_gemv": lambda: lib.ls_gemv(None, 0, 2, 2, p, 2, None, p, p),
        "ls_gemv_timed": lambda: lib.ls_gemv_timed(None, 0, 2, 2, p, 2, None, p, p, 1,
                                                   ctypes.byref(ctypes.c_double())),
        "ls_quantize": lambda: lib.ls_quantize(None, 1, 2, 2, p, 2, p, 2, None),
        "ls_split_f64": lambda: lib.ls_split_f64(None, 2, 2, p, 2, p, 4),
        "ls_selftest_waits": lambda: lib.ls_selftest_waits(None, 0),
        "ls_autotune": lambda: lib.ls_autotune(None, None, 0),
    }


def test_null_context_is_an_argument_error(lslib):
    """A NULL context or server is refused with LS_ERR_ARG before any CUDA call
    (no crash, no device touched); the launch counter of no context is 0."""
    calls = _null_context_calls(lslib)
    declared = set(_declared()) - {"ls_opts_default", "ls_create", "ls_destroy", "ls_strerror",
                                   "ls_kernel_launches", "ls_gemv_noalloc", "ls_tune_load",
                                   "ls_tune_reset", "ls_tune_lookup"}
    assert set(calls) == declared
    for name, call in calls.items():
        assert call() == binding.LS_ERR_ARG, name
    assert lslib.ls_kernel_launches(None) == 0
