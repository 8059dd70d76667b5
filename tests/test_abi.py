"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/cheesegpu.h declares; argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

import paper_2502_11602_gb300 as cg

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "cheesegpu.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cg_status|const char\*|uint64_t)\s+(cg_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_header_symbols():
    lib = cg.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in cheesegpu.h but not exported"
    assert set(names) <= set(cg.EXPORTS) | set(names)
    assert "sm_103a" in cg.cg_version()


def test_build_flags_target_sm_103a():
    from paper_2502_11602_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_argument_errors_without_gpu():
    lib = cg.load()
    h = ctypes.c_void_p()
    # NULL output handle
    assert lib.cg_build(None, 10, 1.0, 1.0, 2, 0, 1, None, None) == 1
    # NULL points
    assert lib.cg_build(None, 10, 1.0, 1.0, 2, 0, 1, None, ctypes.byref(h)) == 1
    assert b"NULL" in lib.cg_last_error()
    fake = ctypes.c_void_p(16)  # never dereferenced: argument checks fail first
    assert lib.cg_build(fake, 0, 1.0, 1.0, 2, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.cg_build(fake, 10, -1.0, 1.0, 2, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.cg_build(fake, 10, float("nan"), 1.0, 2, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.cg_build(fake, 10, 1.0, 1.0, 4, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.cg_build(fake, 10, 1.0, 1.0, 2, 9, 1, None, ctypes.byref(h)) == 1
    assert lib.cg_build(fake, 10, 1.0, 1.0, 2, 0, 7, None, ctypes.byref(h)) == 1
    # allocator hook needs both functions
    assert lib.cg_set_allocator(fake, None, None) == 1
    assert lib.cg_set_allocator(None, None, None) == 0
    # NULL index
    assert lib.cg_index_free(None) == 1
    assert lib.cg_all_points_count(None, 1.0, 0, fake, None, None) == 1
    # the one-call search into a buffer: NULL index, NULL outputs, a
    # negative capacity, a NULL buffer with a positive capacity
    tot = ctypes.c_int64(-1)
    assert lib.cg_radius_search_into(None, fake, 1, 1.0, 0, fake, fake, 10, ctypes.byref(tot), None) == 1
    assert lib.cg_radius_search_into(fake, fake, 1, 1.0, 0, None, fake, 10, ctypes.byref(tot), None) == 1
    assert lib.cg_radius_search_into(fake, fake, 1, 1.0, 0, fake, fake, 10, None, None) == 1
    assert lib.cg_radius_search_into(fake, fake, 1, 1.0, 0, fake, None, 10, ctypes.byref(tot), None) == 1
    assert lib.cg_radius_search_into(fake, fake, 1, 1.0, 0, fake, fake, -1, ctypes.byref(tot), None) == 1
    assert b"capacity" in lib.cg_last_error()
    assert tot.value == -1  # untouched on an argument error
