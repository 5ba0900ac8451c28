"""Host-side failure detection without a GPU: an injected device-allocation
failure inside sfft_plan is reported as SFFT_ERR_NOMEM with its cause, no
allocation is left behind, and the status precedence puts a timed-out wait
before the singular / non-finite symptoms it causes (the mapping is checked
in the source: the GPU test in test_gpu_failure.py exercises it)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_08593_gb300 import binding, build
    build.build()
    return binding.load()


def test_injected_allocation_failure_reports_nomem_and_leaks_nothing(lib, monkeypatch):
    from paper_2603_08593_gb300 import binding
    before = lib.sfft_debug_live_allocations()
    monkeypatch.setenv("SFFT_FAIL_ALLOC", "1")
    desc = binding.Desc(64, 64, 5, 1, 1, 1, binding.PREC["mixed"], 0, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    st = lib.sfft_plan(ctypes.byref(desc), None, ctypes.byref(h))
    assert st == binding.SFFT_ERR_NOMEM
    assert h.value is None
    assert b"injected device allocation failure (SFFT_FAIL_ALLOC=1)" in lib.sfft_last_error()
    assert lib.sfft_debug_live_allocations() == before


def test_timeout_status_takes_precedence():
    src = open(os.path.join(ROOT, "paper_2603_08593_gb300", "csrc", "kernels_solve.cu")).read()
    m = re.search(r"info\[c\] = (.*?);", src, flags=re.S)
    expr = " ".join(m.group(1).split())
    # bit 4 (a wait that gave up) is tested before bits 2 (non-finite) and 1 (singular)
    assert expr.index("s & 4") < expr.index("s & 2") < expr.index("s & 1"), expr
