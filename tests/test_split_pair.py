"""The FP32-pair split that forms the solvers' copy of A (hi = fp32(a),
lo = fp32(a - hi), both to nearest) works on the bit pattern with integer
operations for the common exponent range.  This host check compiles that
code with the system C++ compiler and compares it, bit for bit, with the
plain conversions on random bit patterns, every binary exponent around the
fast range's borders, the rounding ties and carries of the 29 dropped bits,
zeros, subnormals, infinities and NaN.  The device build of the same code is
checked against CUDA's own conversions in test_gpu_gemv.py."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]


def test_split_pair_bits_match_plain_conversions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "split_pair_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off",
                    "-I", str(ROOT / "paper_1511_07207_gb300" / "csrc"),
                    str(ROOT / "tests" / "split_pair_check.cpp"), "-o", str(exe)], check=True)
    p = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stdout
    assert "mismatches 0" in p.stdout
