"""The split epilogue's integer construction of a double from a double-float pair
(csrc/pair2d.cuh, compiled here for the host): bitwise equal to the correctly rounded
h 2^sc + l 2^sc over random pairs, low words far below the high word's last bit (rounding and
sticky bits), ties to even, borrows at powers of two and signed zeros."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pair_to_double_is_correctly_rounded(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "pair2d_test")
    src = os.path.join(ROOT, "tests", "c", "pair2d_test.cpp")
    inc = os.path.join(ROOT, "paper_2311_18715_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", inc, "-o", exe, src], check=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "0 mismatches" in res.stdout
