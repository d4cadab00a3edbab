"""The adjoint's bucket sums round every term to a 64-bit integer with integer
instructions (mls::to_fixed, host-and-device code): checked on the host
against the exact rounding of v 2^s, ties to even, on random floats at the
scales the bucket sum uses, every tie position and the subnormals."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_to_fixed_matches_exact_rounding(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fixed_point_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2401_03365_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fixed_point_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe), "2000000"], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("mismatches 0")
    assert int(out.stdout.split()[1]) > 2_000_000
