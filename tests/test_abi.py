"""The C-ABI library builds for sm_103a and exports every function declared
in include/*.h (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", src):
            name = m.group(1)
            if name.startswith(("sfft_", "rb_", "rbri_", "phot_")) and not name.endswith("_t"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_2603_08593_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ["sfft_plan", "sfft_build_normal", "sfft_solve", "sfft_apply", "sfft_workspace_bytes"]:
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(built_lib):
    from paper_2603_08593_gb300 import binding
    assert set(declared_functions()) <= set(binding.SIGNATURES) | set(getattr(binding, "RB_SIGNATURES", {}))


def test_status_strings_and_arg_errors_without_gpu(built_lib):
    from paper_2603_08593_gb300 import binding
    lib = binding.load()
    assert lib.sfft_status_str(0) == b"ok"
    assert lib.sfft_status_str(7).startswith(b"unsupported")
    # invalid descriptors are rejected on the host before any device work
    h = ctypes.c_void_p()
    for desc in [binding.Desc(64, 64, 4, 1, 1, 1, 1, 0, 0, 0, 0),      # even L
                 binding.Desc(64, 64, 13, 1, 1, 1, 1, 0, 0, 0, 0),     # L too large
                 binding.Desc(64, 64, 5, 3, 3, 1, 1, 0, 0, 0, 0),      # degree above 2
                 binding.Desc(64, 4096, 5, 1, 1, 1, 1, 0, 0, 0, 0)]:   # W too large
        assert lib.sfft_plan(ctypes.byref(desc), None, ctypes.byref(h)) == binding.SFFT_ERR_UNSUPPORTED
    bad = binding.Desc(0, 64, 5, 1, 1, 1, 1, 0, 0, 0, 0)
    assert lib.sfft_plan(ctypes.byref(bad), None, ctypes.byref(h)) == binding.SFFT_ERR_ARG
    unknown_flag = binding.Desc(64, 64, 5, 1, 1, 1, 1, 0, 0, 0, 0, 32)
    assert lib.sfft_plan(ctypes.byref(unknown_flag), None, ctypes.byref(h)) == binding.SFFT_ERR_ARG
    assert lib.sfft_build_normal(None, None, None, None, None, None, None, None) == binding.SFFT_ERR_ARG
