"""The grid sorts points by the Hilbert index of their level-0 cell
(mls::hilbert3, host-and-device code); the search needs every cell of every
level to be one run of consecutive keys.  Checked on the host: bijection,
the level (prefix) property and face-adjacent steps on small grids, the
prefix property on random cells of the full 21-bit grid."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_hilbert_key_properties(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "hilbert_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2401_03365_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "hilbert_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "failures 0"
