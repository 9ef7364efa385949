"""The library's integer-arithmetic binary64 addition (used for the operand sums of
Strassen staging, off the FP64 pipe) against the hardware addition of the host CPU:
bit-identical results on random and edge-case pairs (no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_int_fadd_is_bit_identical_to_hardware_addition(tmp_path):
    exe = tmp_path / "int_fadd_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_1605_01078_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "int_fadd_check.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe), "1000000"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "mismatches 0" in out.stdout
