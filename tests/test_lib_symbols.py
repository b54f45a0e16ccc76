"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/love.h declares (no compute call: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "love.h")).read()
    return sorted(set(re.findall(r"LOVE_API\s+[\w\s\*]+?\b((?:ski|love)_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1803_06058_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in ("ski_build", "love_precompute", "love_predict_mean_var", "love_sample",
                 "love_var_backward"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1803_06058_gb300 import _lib
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_only_declared_symbols_are_exported(lib):
    import subprocess
    from paper_1803_06058_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(_declared())


def test_status_strings_without_gpu(lib):
    assert lib.love_status_string(0) == b"ok"
    assert b"grid" in lib.love_status_string(2)
    assert lib.love_version().startswith(b"love-gb300")


def test_argument_errors_are_returned_synchronously(lib):
    import ctypes as C
    from paper_1803_06058_gb300 import _lib
    h = C.c_void_p()
    assert lib.ski_build(None, None, None, None, C.byref(h)) == 1          # LOVE_ERR_ARG
    d = _lib.love_ski_desc()
    d.dim = 4
    assert lib.ski_build(C.byref(d), C.c_void_p(16), None, None, C.byref(h)) == 1
    assert lib.love_predict_mean_var(None, 10, None, None, None, None) == 1
