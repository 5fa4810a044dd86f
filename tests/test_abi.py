"""The C-ABI library loads and exports every function include/zoom.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zoom.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:zoom_status|void|const char\s*\*)\s+(zoom_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1004_3980_gb300 import build
    build.build()
    from paper_1004_3980_gb300 import capi
    return capi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("zoom_build_dictionary", "zoom_build_index", "zoom_upscale", "zoom_query",
                 "zoom_reconstruct", "zoom_backproject"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1004_3980_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (zoom_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_covers_the_header():
    from paper_1004_3980_gb300 import capi
    assert sorted(capi.SIGNATURES) == declared_functions()


def test_status_strings(lib):
    assert lib.zoom_status_string(0) == b"ok"
    assert lib.zoom_status_string(1) == b"invalid argument"
    assert lib.zoom_status_string(99) == b"unknown status"


def test_null_arguments_are_rejected_on_host(lib):
    from paper_1004_3980_gb300 import capi
    out = C.c_void_p()
    assert lib.zoom_build_index(None, None, None, None, None, C.byref(out)) == 1
    assert b"NULL" in lib.zoom_last_error()
    assert lib.zoom_upscale(None, None, 4, 4, 2, None, None, None) == 1
    assert lib.zoom_query(None, None, 4, 4, None, None, None, None, None, None, None, None) == 1
    assert lib.zoom_ctx_create(0, None, None) == 1
    assert lib.zoom_get_stats(None, None, None) == 1
    p = capi.UpscaleParams(8, 1e-3, 5, 1.5, 0.1, 3, 0, 4, 1e6)
    assert lib.zoom_backproject(None, None, None, 4, 4, C.byref(p), None, None) == 1
    assert lib.zoom_sample_crops(None, None, None, None, 1, None, 1, 4, 4, None, None, None) == 1
