"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports
every function that include/ie.h declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ie_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1512_06126_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ie_setup", "ie_matvec", "ie_solve", "ie_adjoint_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1512_06126_gb300 import ie
    assert set(ie.EXPORTS) <= set(declared_functions())


def test_status_strings(lib):
    lib.ie_status_str.restype = ctypes.c_char_p
    lib.ie_status_str.argtypes = [ctypes.c_int]
    assert lib.ie_status_str(0) == b"ok"
    assert lib.ie_status_str(-2) == b"invalid geometry"


def test_setup_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_1512_06126_gb300 import ie
    L = ie.load()
    out = ctypes.c_void_p()
    # null grid -> IE_ERR_ARG before any device call
    assert L.ie_setup(None, None, None, 1, None, None, 1, None, ctypes.byref(out)) == -1
    assert out.value is None
