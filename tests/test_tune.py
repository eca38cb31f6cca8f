"""The batched engine's tile-shape cache (no GPU): ls_tune_load reads the JSON
cache that ls_autotune writes, ls_tune_lookup returns the choice for a system
from its size bucket [2^b, 2^(b+1)), its padded width sp and the SM count,
and falls back to the defaults (512 columns per task, tensor cores for
sp >= 16) for a missing entry, another GPU's SM count, or after
ls_tune_reset.  Malformed files are refused and leave the choices as they
were."""
import json

import pytest

from paper_1511_07207_gb300 import binding as B


def _write(tmp_path, obj, name="tune.json"):
    p = tmp_path / name
    p.write_text(obj if isinstance(obj, str) else json.dumps(obj))
    return str(p)


CACHE = {"format": "ls-tune-1", "sms": 152, "precision": "fp32", "entries": [
    {"bucket": 10, "sp": 32, "ks32": 1024, "tc": 0, "ms": 1.0},
    {"bucket": 10, "sp": 16, "ks32": 256, "tc": 1, "ms": 1.0},
    {"bucket": 6, "sp": 4, "ks32": 256, "tc": 0, "ms": 1.0},
    {"bucket": 13, "sp": 8, "ks32": 1024, "tc": 0, "ms": 1.0},
]}


@pytest.fixture(autouse=True)
def _reset(lslib, monkeypatch):
    monkeypatch.delenv("LS_ENGINE_TC", raising=False)
    B.ls_tune_reset()
    yield
    B.ls_tune_reset()


def test_defaults_without_a_cache():
    for n, s, tc in [(64, 1, 0), (1000, 8, 0), (1500, 9, 1), (3000, 32, 1), (8192, 20, 1)]:
        assert B.ls_tune_lookup(n, s, 152) == (B.LS_OK, 512, tc)


def test_lookup_by_bucket_width_and_sm_count(tmp_path):
    assert B.ls_tune_load(_write(tmp_path, CACHE)) == B.LS_OK
    # bucket 10 = [1024, 2048); s 17..32 -> sp 32, s 9..16 -> sp 16
    assert B.ls_tune_lookup(1024, 17, 152) == (B.LS_OK, 1024, 0)
    assert B.ls_tune_lookup(2047, 32, 152) == (B.LS_OK, 1024, 0)
    assert B.ls_tune_lookup(1500, 9, 152) == (B.LS_OK, 256, 1)
    assert B.ls_tune_lookup(2048, 32, 152) == (B.LS_OK, 512, 1)     # bucket 11: no entry
    assert B.ls_tune_lookup(1023, 32, 152) == (B.LS_OK, 512, 1)     # bucket 9: no entry
    # sizes below 64 and above 8191 fall into the end buckets
    assert B.ls_tune_lookup(3, 2, 152) == (B.LS_OK, 256, 0)
    assert B.ls_tune_lookup(8192, 5, 152) == (B.LS_OK, 1024, 0)
    # timed on another GPU: defaults
    assert B.ls_tune_lookup(1500, 20, 148) == (B.LS_OK, 512, 1)


def test_reset_and_reload(tmp_path):
    path = _write(tmp_path, CACHE)
    assert B.ls_tune_load(path) == B.LS_OK
    assert B.ls_tune_lookup(1500, 20, 152)[1] == 1024
    B.ls_tune_reset()
    assert B.ls_tune_lookup(1500, 20, 152) == (B.LS_OK, 512, 1)
    assert B.ls_tune_load(path) == B.LS_OK
    assert B.ls_tune_lookup(1500, 20, 152)[1] == 1024


def test_environment_override_of_the_product_form(tmp_path, monkeypatch):
    assert B.ls_tune_load(_write(tmp_path, CACHE)) == B.LS_OK
    monkeypatch.setenv("LS_ENGINE_TC", "0")
    assert B.ls_tune_lookup(1500, 9, 152) == (B.LS_OK, 256, 0)
    monkeypatch.setenv("LS_ENGINE_TC", "2")       # bit 1: sp = 32 only
    assert B.ls_tune_lookup(1500, 20, 152) == (B.LS_OK, 1024, 1)
    assert B.ls_tune_lookup(1500, 9, 152) == (B.LS_OK, 256, 0)


@pytest.mark.parametrize("bad", [
    "", "not json", '{"format": "other", "sms": 152, "entries": []}',
    '{"format": "ls-tune-1", "entries": []}',                                        # no SM count
    '{"format": "ls-tune-1", "sms": 152, "entries": [{"bucket": 10, "sp": 32}]}',   # fields missing
    '{"format": "ls-tune-1", "sms": 152, "entries": [{"bucket": 10, "sp": 12, "ks32": 512, "tc": 0}]}',
    '{"format": "ls-tune-1", "sms": 152, "entries": [{"bucket": 10, "sp": 32, "ks32": 500, "tc": 0}]}',
    '{"format": "ls-tune-1", "sms": 152, "entries": [{"bucket": 10, "sp": 8, "ks32": 512, "tc": 1}]}',
    '{"format": "ls-tune-1", "sms": 152, "entries": [{"bucket": 30, "sp": 8, "ks32": 512, "tc": 0}]}',
])
def test_malformed_caches_are_refused(tmp_path, bad):
    assert B.ls_tune_load(_write(tmp_path, CACHE, "good.json")) == B.LS_OK
    assert B.ls_tune_load(_write(tmp_path, bad)) == B.LS_ERR_ARG
    assert B.ls_tune_lookup(1500, 20, 152) == (B.LS_OK, 1024, 0)    # unchanged


def test_missing_file_and_bad_arguments(tmp_path):
    assert B.ls_tune_load(str(tmp_path / "none.json")) == B.LS_ERR_ARG
    lib = B.load()
    ks, tc = B.ctypes.c_int(), B.ctypes.c_int()
    assert lib.ls_tune_lookup(0, 1, 152, B.ctypes.byref(ks), B.ctypes.byref(tc)) == B.LS_ERR_ARG
    assert lib.ls_tune_lookup(10, 33, 152, B.ctypes.byref(ks), B.ctypes.byref(tc)) == B.LS_ERR_ARG
    assert lib.ls_tune_lookup(10, 1, 0, B.ctypes.byref(ks), B.ctypes.byref(tc)) == B.LS_ERR_ARG
    assert lib.ls_tune_lookup(10, 1, 152, None, B.ctypes.byref(tc)) == B.LS_ERR_ARG
