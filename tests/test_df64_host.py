"""Double-float arithmetic (compute type of complex128 states) checked on the
host: the same header the kernels include, compiled as plain C++, against
IEEE double on 200k seeded random operands.  Bounds: about 2^-47 relative for
conversions, products and fused multiply-adds (relative to the operands'
magnitude for sums), far below the 1e-10 accuracy target of complex128."""

import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_df64_conversion_and_arithmetic_error_bounds(tmp_path):
    exe = tmp_path / "df64_check"
    src = os.path.join(ROOT, "tests", "df64_check.cpp")
    inc = os.path.join(ROOT, "paper_2403_02512_gb300", "csrc")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + inc, src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = dict(zip(out[0::2], out[1::2]))
    assert float(vals["conv"]) < 2.0 ** -46
    assert float(vals["add"]) < 2.0 ** -45
    assert float(vals["mul"]) < 2.0 ** -45
    assert float(vals["fma"]) < 2.0 ** -44
    assert float(vals["rot"]) < 2.0 ** -44
    assert float(vals["fastconv"]) < 2.0 ** -46     # stream conversions (split, join)
    assert float(vals["zero"]) == 0.0
