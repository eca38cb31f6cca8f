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
