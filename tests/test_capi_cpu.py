"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/mls.h declares (no device calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2401_03365_gb300 import build
    return build.build()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "mls.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mls_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_names(libpath):
    from paper_2401_03365_gb300 import capi
    assert _declared_functions() == sorted(capi.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in _declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_reports_status_strings(libpath):
    from paper_2401_03365_gb300 import capi
    lib = capi.lib()
    for name in capi.EXPORTED_SYMBOLS:
        assert hasattr(lib, name)
    assert capi.mls_status_str(0) == "ok"
    assert capi.mls_status_str(-2) == "k too large"
    assert capi.mls_status_str(-999) == "unknown status"
